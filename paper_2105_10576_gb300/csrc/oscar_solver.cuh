// Orchestration of the OSCAR steps (Maes & Menke, arXiv 2105.10576,
// Sections 2.2, 3.1, 3.2) as CUDA graphs.
//
// Each API call (drag step, relaxation, standard step) launches one
// instantiated graph and synchronises once. Inside the graph every pressure
// solve is a conditional WHILE node whose body ends in a one-thread control
// kernel, and the relaxation loop is an outer WHILE node whose control kernel
// applies the paper's early exit (E_k < tol or k = N) on the device. The
// mixed path nests an FP32 PCG (FP64 dot products) inside an FP64
// defect-correction WHILE loop. Graphs are captured from the same launch
// sequence the eager mode issues, and rebuilt when the time step changes.
#pragma once
#include <stdlib.h>
#include <string.h>

#include "oscar_kernels.cuh"

namespace oscar {

#define OSCAR_LAUNCH_CHECK()                                                                              \
    do {                                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                                              \
        if (e_ != cudaSuccess) {                                                                          \
            fprintf(stderr, "oscar: CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return OSCAR_E_CUDA;                                                                          \
        }                                                                                                 \
    } while (0)

#define OSCAR_TRY(x)              \
    do {                          \
        int rc_ = (x);            \
        if (rc_) return rc_;      \
    } while (0)

inline int nblk(long long n) { return (int)((n + BS - 1) / BS); }

// Kernel launch with programmatic stream serialization: the next kernel's
// launch overlaps the tail of this one (each kernel waits in griddep_wait()).
template <typename... KArgs, typename... Args>
inline void launchk(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (Profiler *P = t_prof) {   // in-step timing (eager steps only; never while capturing)
        int slot = prof_begin(P, st, (const void *)kern, grid, block);
        cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
        prof_end(P, st, slot);
    } else {
        cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
    }
}

// ---------------------------------------------------------------------------
// control kernels (one thread). The other loop decisions are taken by the
// finishing block of the reductions (see k_cg_init, k_cg_update,
// k_relax_accum).
// ---------------------------------------------------------------------------
static __global__ void k_inner_start(double *scal, int *ctl, cudaGraphConditionalHandle h) {
    griddep_wait();
    scal[S_RZ0] = 0.0;
    ctl[C_IT] = 0;
    set_cond(ctl, h, true);
}

static __global__ void k_relax_init(int *ctl, cudaGraphConditionalHandle h) {
    griddep_wait(); set_cond(ctl, h, ctl[C_N] > 0); }

// ---------------------------------------------------------------------------
// capture helpers
// ---------------------------------------------------------------------------
inline int cond_handle(Instance &I, cudaGraphConditionalHandle *h) {
    if (!I.capturing) { *h = 0; return 0; }
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    if (cudaStreamGetCaptureInfo(I.stream, &st, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
        return OSCAR_E_CUDA;
    if (cudaGraphConditionalHandleCreate(h, g, 0, 0) != cudaSuccess) return OSCAR_E_CUDA;
    return 0;
}

// Append a WHILE node at the capture point of I.stream and redirect I.stream
// to capture its body.
inline int begin_while(Instance &I, cudaGraphConditionalHandle h, cudaStream_t *saved) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(I.stream, &st, nullptr, &g, &deps, &ed, &nd) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
        return OSCAR_E_CUDA;
    // cudaGraphNodeParams has no default constructor in C++: zero-initialised storage
    alignas(cudaGraphNodeParams) unsigned char buf[sizeof(cudaGraphNodeParams)];
    memset(buf, 0, sizeof(buf));
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(buf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, ed, nd, &np) != cudaSuccess) return OSCAR_E_CUDA;
    if (cudaStreamUpdateCaptureDependencies(I.stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
        cudaSuccess)
        return OSCAR_E_CUDA;
    if (I.depth + 1 >= 4) return OSCAR_E_CUDA;
    cudaStream_t side = I.side[++I.depth];
    if (cudaStreamBeginCaptureToGraph(side, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return OSCAR_E_CUDA;
    *saved = I.stream;
    I.stream = side;
    return 0;
}

inline int end_while(Instance &I, cudaStream_t saved) {
    cudaGraph_t body;
    cudaError_t e = cudaStreamEndCapture(I.stream, &body);
    I.stream = saved;
    --I.depth;
    return e == cudaSuccess ? 0 : OSCAR_E_CUDA;
}

// Read the control words back (eager mode only).
inline int read_ctl(Instance &I) {
    if (cudaMemcpyAsync(I.ctl_host, I.ctl, C_COUNT * sizeof(int), cudaMemcpyDeviceToHost, I.stream) != cudaSuccess)
        return OSCAR_E_CUDA;
    return sync_bounded(I.stream, kSyncTimeoutSec);
}

// while (ctl[C_COND]) body(): a conditional WHILE node when capturing, a host
// loop (one read-back per trip) in eager mode. The decision is written by the
// kernel issued just before the loop and by the last kernel of the body.
template <class F> int loop_while(Instance &I, cudaGraphConditionalHandle h, F body) {
    if (I.capturing) {
        cudaStream_t saved;
        int rc = begin_while(I, h, &saved);
        if (rc) return rc;
        rc = body();
        int rc2 = end_while(I, saved);
        return rc ? rc : rc2;
    }
    for (;;) {
        int rc = read_ctl(I);
        if (rc) return rc;
        if (!I.ctl_host[C_COND]) return 0;
        rc = body();
        if (rc) return rc;
    }
}

template <typename T> struct Impl {
    using M = T;
    using V = T;
    static T *tp(void *p) { return (T *)p; }
    static C3<T> c3(void *const *p) { C3<T> r; for (int a = 0; a < 3; ++a) r.a[a] = (const T *)p[a]; return r; }
    static C3<double> w64(const Instance &I) {
        C3<double> r;
        for (int a = 0; a < 3; ++a) r.a[a] = I.cf64[a];
        return r;
    }
    // FP64 copy of the level-0 coefficients of direction a (mixed path only)
    static double *cf64_out(Instance &I, int a) { return sizeof(T) == sizeof(double) ? nullptr : I.cf64[a]; }
    static P3<T> p3(void *const *p) { P3<T> r; for (int a = 0; a < 3; ++a) r.a[a] = (T *)p[a]; return r; }
    static double *part(Instance &I, int slot) { return I.partials + (size_t)slot * I.red_stride; }


    // --- transport (Eq. alphaExp) ------------------------------------------
    template <int DIM>
    static int transport_d(Instance &I, void *const *phi, double dt) {
        GridD g = to_dev(I.g);
        L3 L = launch3(I.g);
        T rV = (T)(dt / I.g.V);
        launchk(k_transport_low<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, tp(I.alpha), c3(phi), c3(I.nf),
                                                                  (T)I.P.c_alpha, (T)I.P.alpha_inlet, rV, tp(I.aL),
                                                                  tp(I.Pp), tp(I.Pm)), ++I.nlaunch;
        launchk(k_transport_ratio<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, tp(I.alpha), tp(I.aL), tp(I.Pp),
                                                                    tp(I.Pm), rV, tp(I.Rp), tp(I.Rm)), ++I.nlaunch;
        launchk(k_transport_update<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, tp(I.alpha), c3(phi), c3(I.nf),
                                                                     (T)I.P.c_alpha, tp(I.aL), tp(I.Rp), tp(I.Rm), rV,
                                                                     tp(I.alpha_new)), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return 0;
    }
    static int transport(Instance &I, void *const *phi, double dt) {
        return I.g.dim == 3 ? transport_d<3>(I, phi, dt) : transport_d<2>(I, phi, dt);
    }

    // --- interface (Section 2.1) -------------------------------------------
    template <int DIM>
    static int interface_d(Instance &I, void *alpha) {
        GridD g = to_dev(I.g);
        L3 L = launch3(I.g);
        void *src = alpha;
        for (int pass = 0; pass < I.P.n_smooth; ++pass) {
            void *dst = (pass % 2 == 0) ? I.alpha_s : I.alpha_tmp;
            launchk(k_smooth<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, tp(src), tp(dst)), ++I.nlaunch;
            src = dst;
        }
        const T *as = tp(src);
        T ct = (T)I.cos_theta, dn = (T)I.deltaN;
        L3 F0 = launch3_faces(I.g, 0), F1 = launch3_faces(I.g, 1), F2 = launch3_faces(I.g, 2);
        launchk(k_normals<DIM, 0, T>, F0.grid, F0.block, 0, I.stream, g, I.info, as, ct, dn, tp(I.nf[0])), ++I.nlaunch;
        launchk(k_normals<DIM, 1, T>, F1.grid, F1.block, 0, I.stream, g, I.info, as, ct, dn, tp(I.nf[1])), ++I.nlaunch;
        if (DIM == 3)
            launchk(k_normals<DIM, 2, T>, F2.grid, F2.block, 0, I.stream, g, I.info, as, ct, dn, tp(I.nf[2])), ++I.nlaunch;
        launchk(k_curvature<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, c3(I.nf), tp(I.kappa)), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return 0;
    }
    static int interface_(Instance &I, void *alpha) {
        return I.g.dim == 3 ? interface_d<3>(I, alpha) : interface_d<2>(I, alpha);
    }

    // --- multigrid -----------------------------------------------------------
    static MG3<M> mg3(const Level &L) { MG3<M> c; for (int a = 0; a < 3; ++a) c.a[a] = (const M *)L.c[a]; return c; }

    template <int DIM>
    static int mg_coeffs_d(Instance &I) {
        for (int l = 0; l < I.nlev; ++l) {
            Level &L = I.lev[l];
            GridD g = to_dev(L.g);
            L3 LL = launch3(L.g);
            if (l == 0) {
                launchk(k_mg_diag<DIM, M>, LL.grid, LL.block, 0, I.stream, g, L.fluid, mg3(L), (M *)L.diag,
                        (M *)L.idiag), ++I.nlaunch;
            } else {
                Level &F = I.lev[l - 1];
                P3<M> cc;
                for (int a = 0; a < 3; ++a) cc.a[a] = (M *)L.c[a];
                launchk(k_mg_level_operator<DIM, M>, LL.grid, LL.block, 0, I.stream, to_dev(F.g), g, F.r[0], F.r[1],
                        F.r[2], mg3(F), cc, (const uint8_t *)L.fluid, (M *)L.diag, (M *)L.idiag), ++I.nlaunch;
            }
        }
        {   // the coarse CTA's shared-memory image for this set of coefficients
            CLevels<M> P;
            cta_levels(I, P, I.lc0);
            launchk(k_mg_coarse_pack<DIM, M>, 1, kCtaThreads, I.cta_img_bytes, I.stream, P, (uint4 *)I.cta_img,
                    (int)(I.cta_img_bytes / 16), I.ctl), ++I.nlaunch;
        }
        OSCAR_LAUNCH_CHECK();
        return 0;
    }

    // levels l0.. of the single-CTA coarse kernel with their shared-memory
    // layout; returns the bytes of shared memory they need
    static size_t cta_levels(Instance &I, CLevels<M> &P, int l0, size_t base = 0, bool allow_exact = true) {
        memset(&P.G, 0, sizeof(P.G));
        P.n = I.nlev - l0;
        P.exact = 0;
        P.oinv = 0;
        P.refresh = I.coarse_refresh;
        if (allow_exact)   // stop at the first level small enough for an exact solve
            for (int q = 0; q < P.n; ++q)
                if (I.lev[l0 + q].g.ncell <= kExactCells) { P.n = q + 1; P.exact = 1; break; }
        P.nu = I.mg_nu_cta;
        P.nu_top = l0 == 0 ? I.mg_nu : I.mg_nu_cta;
        P.coarse_sweeps = I.mg_coarse_sweeps;
        size_t off = base;
        auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 15) & ~(size_t)15; return (int)o; };
        size_t nmax = 0;
        for (int q = 0; q < P.n && q < kMaxCL; ++q) {
            Level &L = I.lev[l0 + q];
            CLevel<M> &C = P.L[q];
            C.g = to_dev(L.g);
            for (int a = 0; a < 3; ++a) C.c[a] = (const M *)L.c[a];
            C.fluid = L.fluid;
            for (int a = 0; a < 3; ++a) C.r[a] = L.r[a];
            C.rnx = 1.0f / (float)L.g.nx;
            C.rny = 1.0f / (float)L.g.ny;
            C.rhx = 1.0f / (float)((L.g.nx + 1) / 2);
            C.nh = ((L.g.nx + 1) / 2) * L.g.ny * L.g.nz;
            size_t n = L.g.ncell, pad = (size_t)L.g.nx * L.g.ny, dim = L.g.dim;
            nmax = n > nmax ? n : nmax;
            C.ox = take((n + 2 * pad) * sizeof(M)) + (int)(pad * sizeof(M));
            C.ob = take(n * sizeof(M));
            C.od = take(n * sizeof(M));
            C.oi = take(n * sizeof(M));
            C.ow = take(2 * dim * n * sizeof(M));
            C.opk = take(n * sizeof(uint32_t));
            C.ol[0] = take(C.nh * sizeof(unsigned short));
            C.ol[1] = take(C.nh * sizeof(unsigned short));
            C.ofl = take(n);
            for (int a = 0; a < 3; ++a) C.os[a] = take(a < L.g.dim ? (size_t)L.g.nf[a] * sizeof(M) : 0);
        }
        P.ors = take(nmax * sizeof(M));
        if (P.exact) {
            const int ne = I.lev[l0 + P.n - 1].g.ncell;
            P.oinv = take((size_t)ne * ne * sizeof(M));
        }
        return P.n > kMaxCL ? (size_t)-1 : off;
    }

    // the global-coefficient level lg of the coarse CTA, its x and b placed in
    // shared memory after the image of the CTA's levels
    static void gl_fill(Instance &I, CLevels<M> &P, int lg) {
        GLevel<M> &G = P.G;
        const Level &L = I.lev[lg];
        G.active = 1;
        G.g = to_dev(L.g);
        G.c = mg3(L);
        G.diag = (const M *)L.diag;
        G.idiag = (const M *)L.idiag;
        G.fluid = L.fluid;
        for (int a = 0; a < 3; ++a) G.r[a] = L.r[a];
        G.rhx = 1.0f / (float)((L.g.nx + 1) / 2);
        G.rny = 1.0f / (float)L.g.ny;
        const size_t base = (I.cta_img_bytes + 15) & ~(size_t)15;
        G.ox = (int)base;
        G.ob = (int)(base + (((size_t)L.g.ncell * sizeof(M) + 15) & ~(size_t)15));
        G.nu = I.mg_nu_c;
    }
    static size_t gl_bytes(const Instance &I, int lg, size_t img) {
        const size_t n = (size_t)I.lev[lg].g.ncell * sizeof(M);
        return ((img + 15) & ~(size_t)15) + 2 * ((n + 15) & ~(size_t)15);
    }

    // x / b of level l (level 0 works in place on the Krylov vectors z / r)
    static M *lx(Instance &I, int l, V *z) { return l == 0 ? (M *)z : (M *)I.lev[l].x; }
    static M *lb(Instance &I, int l, V *r) { return l == 0 ? (M *)r : (M *)I.lev[l].b; }

    // one half sweep; with_dot (finest level only) also forms r.z and beta
    template <int DIM>
    static void smooth_level(Instance &I, int l, int colour, M *x, const M *b, bool with_dot = false) {
        Level &L = I.lev[l];
        GridD g = to_dev(L.g);
        L3 LL = launch3((L.g.nx + 1) / 2, L.g.ny, L.g.nz);
        if (with_dot)
            launchk(k_mg_rbgs_dot<DIM, M>, LL.grid, LL.block, 0, I.stream, g, mg3(L), (const M *)L.idiag, x, b, colour,
                    I.partials, I.ticket, I.scal), ++I.nlaunch;
        else
            for (int rep = 0; rep < (l == 0 && I.repeat_fine ? 2 : 1); ++rep)   // a repeat is idempotent
                launchk(k_mg_rbgs<DIM, M, false>, LL.grid, LL.block, 0, I.stream, g, mg3(L), (const M *)L.idiag, x,
                        b, colour, g, 0, 0, 0, (const M *)nullptr), ++I.nlaunch;
    }
    // the first post-smoothing half sweep (colour 1) of level l with the
    // prolongation from level l + 1 (x of level l + 1 in xc) folded in
    template <int DIM>
    static void prolong_smooth(Instance &I, int l, M *x, const M *b, const M *xc) {
        Level &L = I.lev[l], &C = I.lev[l + 1];
        GridD g = to_dev(L.g), gc = to_dev(C.g);
        L3 LL = launch3((L.g.nx + 1) / 2, L.g.ny, L.g.nz);
        launchk(k_mg_rbgs<DIM, M, true>, LL.grid, LL.block, 0, I.stream, g, mg3(L), (const M *)L.idiag, x, b, 1, gc,
                L.r[0] >> 1, L.r[1] >> 1, L.r[2] >> 1, xc), ++I.nlaunch;
    }

    template <int DIM, int RX, int RY, int RZ>
    static void rr_launch(Instance &I, const Level &L, const Level &C, const M *x, const M *b, M *bc, M *xc, int first) {
        using TT = RRTile<DIM>;
        const dim3 grid((L.g.nx + TT::X - 1) / TT::X, (L.g.ny + TT::Y - 1) / TT::Y, (L.g.nz + TT::Z - 1) / TT::Z);
        launchk(k_mg_resid_restrict<DIM, M, RX, RY, RZ>, grid, dim3(TT::X, TT::Y, TT::Z), 0, I.stream, to_dev(L.g),
                to_dev(C.g), L.fluid, mg3(L), (const M *)L.diag, x, b, bc, xc, (const M *)C.idiag, first);
        ++I.nlaunch;
    }
    // fused residual + restriction (+ the coarse level's first colour-0 half
    // sweep when first is set), dispatched on the coarsening ratios
    template <int DIM>
    static void resid_restrict(Instance &I, const Level &L, const Level &C, const M *x, const M *b, M *bc, M *xc,
                               int first) {
        int code = (L.r[0] == 2) | ((L.r[1] == 2) << 1) | ((L.r[2] == 2) << 2);
        switch (code) {
            case 1: rr_launch<DIM, 2, 1, 1>(I, L, C, x, b, bc, xc, first); break;
            case 2: rr_launch<DIM, 1, 2, 1>(I, L, C, x, b, bc, xc, first); break;
            case 3: rr_launch<DIM, 2, 2, 1>(I, L, C, x, b, bc, xc, first); break;
            case 4: rr_launch<DIM, 1, 1, 2>(I, L, C, x, b, bc, xc, first); break;
            case 5: rr_launch<DIM, 2, 1, 2>(I, L, C, x, b, bc, xc, first); break;
            case 6: rr_launch<DIM, 1, 2, 2>(I, L, C, x, b, bc, xc, first); break;
            case 7: rr_launch<DIM, 2, 2, 2>(I, L, C, x, b, bc, xc, first); break;
            default: rr_launch<DIM, 1, 1, 1>(I, L, C, x, b, bc, xc, first); break;
        }
    }

    // z = V-cycle(r): pre-smoothing red-black, post-smoothing black-red
    // (symmetric, so a valid CG preconditioner); levels from lc0 down run in
    // one CTA. The first colour-0 half sweep of each level above the CTA is
    // done by the kernel that produces its right-hand side (k_cg_init /
    // k_cg_update for the finest level, the restriction for the others).
    template <int DIM>
    static int vcycle_d(Instance &I, V *r, V *z) {
        const int lk = I.lg >= 0 ? I.lg : I.lc0;   // first level not worked by per-level kernels
        for (int l = 0; l < lk; ++l) {
            Level &L = I.lev[l], &C = I.lev[l + 1];
            M *x = lx(I, l, z), *b = lb(I, l, r);
            int nu = l == 0 ? I.mg_nu : I.mg_nu_c;
            for (int s = 0; s < nu; ++s) {
                if (s > 0) smooth_level<DIM>(I, l, 0, x, b);
                smooth_level<DIM>(I, l, 1, x, b);
            }
            resid_restrict<DIM>(I, L, C, x, b, lb(I, l + 1, r), lx(I, l + 1, z), l + 1 < lk ? 1 : 0);
        }
        {
            CLevels<M> P;
            cta_levels(I, P, I.lc0);
            P.b_top = lb(I, I.lc0, r);
            P.x_top = lx(I, I.lc0, z);
            if (I.lg >= 0) {
                gl_fill(I, P, I.lg);
                P.G.b_glob = lb(I, I.lg, r);
                P.G.x_glob = lx(I, I.lg, z);
            }
            launchk(k_mg_coarse<DIM, M>, 1, kCtaThreads, I.cta_smem, I.stream, P, (const uint4 *)I.cta_img,
                    (int)(I.cta_img_bytes / 16)), ++I.nlaunch;
        }
        for (int l = lk - 1; l >= 0; --l) {
            M *x = lx(I, l, z), *b = lb(I, l, r);
            int nu = l == 0 ? I.mg_nu : I.mg_nu_c;
            for (int s = 0; s < nu; ++s) {
                if (s == 0) prolong_smooth<DIM>(I, l, x, b, (const M *)lx(I, l + 1, z));
                else smooth_level<DIM>(I, l, 1, x, b);
                smooth_level<DIM>(I, l, 0, x, b, l == 0 && s == nu - 1);   // the last one also forms r.z
            }
        }
        OSCAR_LAUNCH_CHECK();
        return 0;
    }

    // r = b - M q (FP64), ||b||^2, ||r||^2 into S_BB, S_RR, then the loop
    // decision of residual_control(mode)
    // (with_E: also the normalised residual E_k of Section 3.2 for q, b)
    template <int DIM>
    static void residual64(Instance &I, const double *q, const double *b, int mode, cudaGraphConditionalHandle h,
                           V *zero1, V *zero2, double *r64 = nullptr, bool with_E = false) {
        GridD g = to_dev(I.g);
        L3 L = launch_rows(I.g, kRedBlocks);
        launchk(k_cg_init<DIM, T, V>, L.grid, L.block, 0, I.stream, g, I.info, w64(I), q, b, (V *)I.cg_r, r64,
                (const V *)I.lev[0].idiag, (V *)I.cg_z, zero1, zero2, I.partials, I.red_stride, I.ticket, L.nblocks,
                I.scal, I.ctl, I.P.cg_rtol, mode, h, with_E ? 1.0 / (double)I.n_fluid : 0.0), ++I.nlaunch;
    }

    // one PCG iteration on M x = r with Krylov vectors z, p, Ap (type V)
    template <int DIM>
    static int pcg_body(Instance &I, V *x, int target_slot, cudaGraphConditionalHandle h, int xfresh) {
        GridD g = to_dev(I.g);
        L3 L = launch_rows(I.g, kRedBlocks);
        int n = I.g.ncell;
        V *r = (V *)I.cg_r, *z = (V *)I.cg_z, *p = (V *)I.cg_p, *Ap = (V *)I.cg_Ap;
        long long n0 = I.nlaunch;
        OSCAR_TRY(vcycle_d<DIM>(I, r, z));
        if (I.lc0 == 0)   // the whole V-cycle ran in the coarse CTA: r.z on its own
            launchk(k_cg_dot_rz<V>, kRedBlocks, BS, 0, I.stream, n, r, z, I.partials, I.ticket, I.scal), ++I.nlaunch;
        if constexpr (sizeof(V) == sizeof(float)) {
            L3 LA = launch_rpt(I.g, kApplyRows);
            launchk(k_cg_pz_apply<DIM, T, V, kApplyRows>, LA.grid, LA.block, 0, I.stream, g, I.info, c3(I.lev[0].c),
                    (const V *)z, p, Ap, I.partials, I.ticket, LA.nblocks, I.scal), ++I.nlaunch;
        } else {   // FP64 path: the search direction as written, M p applied directly
            launchk(k_cg_pupdate<V>, kRedBlocks, BS, 0, I.stream, n, I.scal, z, p), ++I.nlaunch;
            launchk(k_cg_apply_dot<DIM, T, V>, L.grid, L.block, 0, I.stream, g, I.info, c3(I.lev[0].c), p, Ap,
                    I.partials, I.ticket, L.nblocks, I.scal), ++I.nlaunch;
        }
        L3 LU = launch_rpt(I.g, kUpdateRows);
        launchk(k_cg_update<V, kUpdateRows>, LU.grid, LU.block, 0, I.stream, g, x, r, p, Ap, (const V *)I.lev[0].idiag,
                z, I.partials, I.ticket, I.scal, I.ctl, I.P.cg_maxit, target_slot, xfresh, h), ++I.nlaunch;
        if (I.capturing) {
            I.n_cg_body = I.nlaunch - n0;
            I.cg_bodies_captured += 1;
        }
        OSCAR_LAUNCH_CHECK();
        return 0;
    }

    // Pressure solve M q = b. FP64 path: PCG on q itself. Mixed path: FP64
    // defect correction around an FP32 PCG for the correction e.
    template <int DIM>
    static int pcg_d(Instance &I, double *q, const double *b, bool with_E) {
        size_t nbytes = (size_t)I.g.ncell * sizeof(V);
        (void)nbytes;
        if constexpr (sizeof(T) == sizeof(double)) {
            cudaGraphConditionalHandle h;
            OSCAR_TRY(cond_handle(I, &h));
            residual64<DIM>(I, q, b, 0, h, (V *)I.cg_p, nullptr, nullptr, with_E);
            return loop_while(I, h, [&]() -> int { return pcg_body<DIM>(I, (V *)q, S_TARGET, h, 0); });
        } else {
        cudaGraphConditionalHandle ho;
        OSCAR_TRY(cond_handle(I, &ho));
        // the inner solve starts e and p from 0 itself (xfresh, beta = 0), so
        // neither is cleared; the FP64 residual is evaluated once, then updated
        // by k_cg_refine at the end of every trip
        residual64<DIM>(I, q, b, 1, ho, nullptr, nullptr, I.cg_r64, with_E);
        return loop_while(I, ho, [&]() -> int {
            long long n0 = I.nlaunch, cg0 = I.cg_bodies_captured;
            cudaGraphConditionalHandle hi;
            OSCAR_TRY(cond_handle(I, &hi));
            launchk(k_inner_start, 1, 1, 0, I.stream, I.scal, I.ctl, hi), ++I.nlaunch;
            OSCAR_TRY(loop_while(I, hi, [&]() -> int { return pcg_body<DIM>(I, (V *)I.cg_e, S_ITARGET, hi, 1); }));
            if constexpr (sizeof(V) == sizeof(float)) {
                GridD g = to_dev(I.g);
                L3 L = launch_rows(I.g, kRedBlocks);
                launchk(k_cg_refine<DIM>, L.grid, L.block, 0, I.stream, g, I.info, c3(I.lev[0].c), (const float *)I.cg_e,
                        q, I.cg_r64, (float *)I.cg_r, (const float *)I.lev[0].idiag, (float *)I.cg_z, I.partials,
                        I.red_stride, I.ticket, L.nblocks, I.scal, I.ctl, I.P.cg_rtol, ho), ++I.nlaunch;
            }
            if (I.capturing) I.n_outer_body = (I.nlaunch - n0) - (I.cg_bodies_captured - cg0) * I.n_cg_body;
            OSCAR_LAUNCH_CHECK();
            return 0;
        });
        }
    }

    // --- PISO (Section 2.2) --------------------------------------------------
    template <int DIM>
    static int piso_d(Instance &I, void *const *v, double *q, void *const *phi, bool has_st, double vin0, double dt) {
        GridD g = to_dev(I.g);
        L3 L = launch3(I.g);
        L3 F[3] = {launch3_faces(I.g, 0), launch3_faces(I.g, 1), launch3_faces(I.g, 2)};
        Fluid<T> fl{(T)I.P.rho1, (T)I.P.rho2, (T)I.P.mu1, (T)I.P.mu2};
        const T *al = tp(I.alpha_new);
        launchk(k_rA<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, al, c3(I.phic), fl, (T)dt, tp(I.rA)), ++I.nlaunch;
        void **cf = I.lev[0].c;
        T sig = (T)I.P.sigma;
        int st = has_st ? 1 : 0;
        launchk(k_face_coeffs<0, T>, F[0].grid, F[0].block, 0, I.stream, g, I.info, tp(I.rA), tp(I.kappa), al, sig, st,
                                                                    tp(cf[0]), tp(I.fst[0]), cf64_out(I, 0)), ++I.nlaunch;
        launchk(k_face_coeffs<1, T>, F[1].grid, F[1].block, 0, I.stream, g, I.info, tp(I.rA), tp(I.kappa), al, sig, st,
                                                                    tp(cf[1]), tp(I.fst[1]), cf64_out(I, 1)), ++I.nlaunch;
        if (DIM == 3)
            launchk(k_face_coeffs<2, T>, F[2].grid, F[2].block, 0, I.stream, g, I.info, tp(I.rA), tp(I.kappa), al, sig, st,
                                                                        tp(cf[2]), tp(I.fst[2]), cf64_out(I, 2)), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        OSCAR_TRY(mg_coeffs_d<DIM>(I));
        P3<T> Gp0 = p3(&I.G[0]), Gp1 = p3(&I.G[3]), Gp2 = p3(&I.G[6]);
        C3<T> Gc0 = c3(&I.G[0]), Gc1 = c3(&I.G[3]), Gc2 = c3(&I.G[6]);
        for (int corr = 0; corr < I.P.n_piso; ++corr) {
            launchk(k_vel_grad<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, c3(v), (T)vin0, Gp0, Gp1, Gp2), ++I.nlaunch;
            launchk(k_momentum_H<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, c3(v), c3(I.vold), c3(I.phic), al,
                                                                   tp(I.rA), fl, (T)vin0, (T)dt, Gc0, Gc1, Gc2,
                                                                   p3(I.hbya)), ++I.nlaunch;
            launchk(k_phistar_rhs<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, c3(I.hbya), tp(I.rA), c3(I.fst),
                    (T)vin0, p3(I.phis), I.cg_b), ++I.nlaunch;
            // E_k, the normalised initial residual of the first corrector
            // (Section 3.2), is formed by the solve's initial-residual kernel
            if (corr == 0)
                launchk(k_sum_to<double>, kRedBlocks, BS, 0, I.stream, g.ncell, q, 1.0, I.partials, I.ticket, I.scal,
                                                                  S_QSUM), ++I.nlaunch;
            OSCAR_LAUNCH_CHECK();
            OSCAR_TRY(pcg_d<DIM>(I, q, I.cg_b, corr == 0));
            launchk(k_correct<DIM, T>, L.grid, L.block, 0, I.stream, g, I.info, c3(I.phis), c3(cf), q, p3(phi),
                    c3(I.hbya), tp(I.rA), c3(I.fst), p3(v)), ++I.nlaunch;
            OSCAR_LAUNCH_CHECK();
        }
        return 0;
    }
    static int piso(Instance &I, void *const *v, double *q, void *const *phi, bool has_st, double vin0, double dt) {
        return I.g.dim == 3 ? piso_d<3>(I, v, q, phi, has_st, vin0, dt) : piso_d<2>(I, v, q, phi, has_st, vin0, dt);
    }

    static int copy_fields(Instance &I, void *const *dst, void *const *src, int is_face) {
        for (int a = 0; a < I.g.dim; ++a) {
            size_t n = is_face ? I.g.nf[a] : I.g.ncell;
            if (cudaMemcpyAsync(dst[a], src[a], n * sizeof(T), cudaMemcpyDeviceToDevice, I.stream) != cudaSuccess)
                return OSCAR_E_CUDA;
        }
        return 0;
    }
    static int sum_faces(Instance &I, void *const *a, void *const *b, void *const *out) {
        for (int d = 0; d < I.g.dim; ++d)
            launchk(k_sum2<T>, nblk(I.g.nf[d]), BS, 0, I.stream, I.g.nf[d], tp(a[d]), tp(b[d]), tp(out[d])), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return 0;
    }
    // scal[slot] = sigma A + kinetic energy of u_cr (the energy exit test)
    static int relax_energy(Instance &I, int slot) {
        GridD g = to_dev(I.g);
        Fluid<T> fl{(T)I.P.rho1, (T)I.P.rho2, (T)I.P.mu1, (T)I.P.mu2};
        if (I.g.dim == 3)
            launchk(k_relax_energy<3, T>, kRedBlocks, BS, 0, I.stream, I.g.ncell, g, I.info, (const T *)I.alpha,
                    c3(I.u_cr), fl, I.P.sigma, I.partials, I.red_stride, I.ticket, I.scal, slot), ++I.nlaunch;
        else
            launchk(k_relax_energy<2, T>, kRedBlocks, BS, 0, I.stream, I.g.ncell, g, I.info, (const T *)I.alpha,
                    c3(I.u_cr), fl, I.P.sigma, I.partials, I.red_stride, I.ticket, I.scal, slot), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return 0;
    }
    static int commit_alpha(Instance &I) {
        return cudaMemcpyAsync(I.alpha, I.alpha_new, (size_t)I.g.ncell * sizeof(T), cudaMemcpyDeviceToDevice,
                               I.stream) == cudaSuccess ? 0 : OSCAR_E_CUDA;
    }
    static int load_ctl(Instance &I) {
        return cudaMemcpyAsync(I.ctl, I.ctl_host, C_COUNT * sizeof(int), cudaMemcpyHostToDevice, I.stream) ==
                       cudaSuccess ? 0 : OSCAR_E_CUDA;
    }

    // --- step bodies ---------------------------------------------------------
    // Section 3.1: viscous-drag step
    static int body_drag(Instance &I, double dt) {
        OSCAR_TRY(load_ctl(I));
        OSCAR_TRY(transport(I, I.phi_vd, dt));
        OSCAR_TRY(sum_faces(I, I.phi_vd, I.phi_cr, I.phic));
        OSCAR_TRY(copy_fields(I, I.vold, I.u_vd, 0));
        OSCAR_TRY(piso(I, I.u_vd, I.p_vd, I.phi_vd, false, I.P.U_inlet, dt));
        OSCAR_TRY(commit_alpha(I));
        return interface_(I, I.alpha);
    }
    // Section 2.2: standard time-stepping
    static int body_standard(Instance &I, double dt) {
        OSCAR_TRY(load_ctl(I));
        OSCAR_TRY(transport(I, I.phi_vd, dt));
        OSCAR_TRY(interface_(I, I.alpha_new));
        OSCAR_TRY(copy_fields(I, I.phic, I.phi_vd, 1));
        OSCAR_TRY(copy_fields(I, I.vold, I.u_vd, 0));
        OSCAR_TRY(piso(I, I.u_vd, I.p_vd, I.phi_vd, true, I.P.U_inlet, dt));
        OSCAR_TRY(commit_alpha(I));
        for (int a = 0; a < I.g.dim; ++a)
            if (cudaMemsetAsync(I.u_sum[a], 0, I.g.ncell * sizeof(double), I.stream) != cudaSuccess)
                return OSCAR_E_CUDA;
        return 0;
    }
    // Section 3.2: relaxation loop with the early exit on the device
    static int body_relax(Instance &I, double dt, long long *n_pre, long long *n_body) {
        long long s0 = I.nlaunch;
        OSCAR_TRY(load_ctl(I));
        for (int a = 0; a < I.g.dim; ++a)
            if (cudaMemsetAsync(I.u_sum[a], 0, I.g.ncell * sizeof(double), I.stream) != cudaSuccess)
                return OSCAR_E_CUDA;
        cudaGraphConditionalHandle h;
        OSCAR_TRY(cond_handle(I, &h));
        const bool area = I.P.conv_mode == OSCAR_CONV_AREA;
        if (area) OSCAR_TRY(relax_energy(I, S_AREA0));
        launchk(k_relax_init, 1, 1, 0, I.stream, I.ctl, h), ++I.nlaunch;
        *n_pre = I.nlaunch - s0;
        long long b0 = I.nlaunch, cg0 = I.cg_bodies_captured;
        long long ob0 = I.cg_bodies_captured;
        int outer_bodies_before = 0;
        (void)ob0;
        (void)outer_bodies_before;
        int npiso_solves = 0;
        int rc = loop_while(I, h, [&]() -> int {
            OSCAR_TRY(transport(I, I.phi_cr, dt));
            OSCAR_TRY(interface_(I, I.alpha_new));
            OSCAR_TRY(sum_faces(I, I.phi_vd, I.phi_cr, I.phic));
            OSCAR_TRY(copy_fields(I, I.vold, I.u_cr, 0));
            OSCAR_TRY(piso(I, I.u_cr, I.p_cr, I.phi_cr, true, 0.0, dt));
            npiso_solves += I.P.n_piso;
            OSCAR_TRY(commit_alpha(I));
            if (area) OSCAR_TRY(relax_energy(I, S_AREA1));
            P3<double> us;
            for (int a = 0; a < 3; ++a) us.a[a] = I.u_sum[a];
            double invU = I.P.U_inlet > 0 ? 1.0 / I.P.U_inlet : 0.0;
            if (I.g.dim == 3)
                launchk(k_relax_accum<3, T>, kRedBlocks, BS, 0, I.stream, I.g.ncell, I.info, c3(I.u_cr), c3(I.vold), us,
                                                                     I.partials, I.ticket, I.scal, I.ctl,
                                                                     I.P.conv_mode, I.P.conv_tol, invU, h), ++I.nlaunch;
            else
                launchk(k_relax_accum<2, T>, kRedBlocks, BS, 0, I.stream, I.g.ncell, I.info, c3(I.u_cr), c3(I.vold), us,
                                                                     I.partials, I.ticket, I.scal, I.ctl,
                                                                     I.P.conv_mode, I.P.conv_tol, invU, h), ++I.nlaunch;
            OSCAR_LAUNCH_CHECK();
            return 0;
        });
        // launches of one sub-step outside the loop bodies of its pressure solves
        long long outer = sizeof(T) == sizeof(double) ? 0 : (long long)npiso_solves * I.n_outer_body;
        *n_body = (I.nlaunch - b0) - (I.cg_bodies_captured - cg0) * I.n_cg_body - outer;
        return rc;
    }

    static int build(Instance &I, int kind, double dt) {
        GraphSlot &G = I.gslot[kind];
        if (G.valid && G.dt == dt) return 0;
        if (G.valid) {
            cudaGraphExecDestroy(G.exec);
            cudaGraphDestroy(G.graph);
            G.valid = 0;
        }
        if (cudaStreamBeginCapture(I.stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return OSCAR_E_CUDA;
        I.capturing = 1;
        I.depth = 0;
        long long s0 = I.nlaunch, cg0 = I.cg_bodies_captured;
        long long n_pre = 0, n_body = 0;
        int rc;
        if (kind == 0) rc = body_drag(I, dt);
        else if (kind == 1) rc = body_relax(I, dt, &n_pre, &n_body);
        else rc = body_standard(I, dt);
        if (kind != 1) {
            long long outer = sizeof(T) == sizeof(double) ? 0 : (long long)I.P.n_piso * I.n_outer_body;
            n_pre = (I.nlaunch - s0) - (I.cg_bodies_captured - cg0) * I.n_cg_body - outer;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(I.stream, &graph);
        I.capturing = 0;
        if (rc || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc ? rc : OSCAR_E_CUDA;
        }
        if (cudaGraphInstantiate(&G.exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            cudaGetLastError();
            return OSCAR_E_CUDA;
        }
        G.graph = graph;
        G.dt = dt;
        G.valid = 1;
        G.n_pre = n_pre;
        G.n_body = n_body;
        return 0;
    }

    // Launch step `kind` (graph, or eager loops) and read its control words back.
    // launch one step (graph, or the eager sequence) and the copies of its
    // device scalars back to the host, without waiting
    static bool eager_now(const Instance &I) { return I.eager || (I.prof && I.prof->enabled); }
    static int run_launch(Instance &I, int kind, double dt, int N) {
        BlockXScope bxs(I.block_x);
        const bool eager = eager_now(I);
        if (!eager) OSCAR_TRY(build(I, kind, dt));
        OSCAR_TRY(sync_bounded(I.stream, kSyncTimeoutSec));   // ctl_host is read by the graph
        for (int q = 0; q < C_COUNT; ++q) I.ctl_host[q] = 0;
        I.ctl_host[C_N] = N;
        if (eager) {
            long long l0 = I.nlaunch, d0 = 0, d1 = 0;
            t_prof = (I.prof && I.prof->enabled) ? I.prof : nullptr;
            int rc = kind == 0 ? body_drag(I, dt) : kind == 1 ? body_relax(I, dt, &d0, &d1) : body_standard(I, dt);
            t_prof = nullptr;
            if (rc) return rc;
            I.nexec += I.nlaunch - l0;
        } else if (cudaGraphLaunch(I.gslot[kind].exec, I.stream) != cudaSuccess) {
            return OSCAR_E_CUDA;
        }
        if (cudaMemcpyAsync(I.scal_host, I.scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, I.stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(I.ctl_host, I.ctl, C_COUNT * sizeof(int), cudaMemcpyDeviceToHost, I.stream) !=
                cudaSuccess)
            return OSCAR_E_CUDA;
        I.pending = kind;
        I.pending_dt = dt;
        I.pending_N = N;
        return 0;
    }
    static int run(Instance &I, int kind, double dt, int N) {
        OSCAR_TRY(run_launch(I, kind, dt, N));
        return run_finish(I);
    }
    // wait for the launched step and account for it
    static int run_finish(Instance &I) {
        const int kind = I.pending;
        const double dt = I.pending_dt;
        I.pending = -1;
        OSCAR_TRY(sync_bounded(I.stream, kSyncTimeoutSec));
        const GraphSlot &G = I.gslot[kind];
        int its = I.ctl_host[C_ITSUM];
        int trips = kind == 1 ? I.ctl_host[C_K] : 1;
        if (!eager_now(I)) {
            long long outer_trips = sizeof(T) == sizeof(double) ? 0 : (long long)I.ctl_host[C_OSUM];
            I.nexec += G.n_pre + (long long)(kind == 1 ? trips : 0) * G.n_body + (long long)its * I.n_cg_body +
                       outer_trips * I.n_outer_body;
        }
        I.cg_iters_last = its;
        I.cg_iters_total += its;
        I.cell_updates += (long long)trips * I.n_fluid;
        I.last_dt = dt;
        if (I.ctl_host[C_NAN]) return OSCAR_E_NAN;
        return I.ctl_host[C_NOTCONV] ? OSCAR_E_NOT_CONVERGED : 0;
    }
};

template <typename T> void Solver<T>::release_graphs(Instance &I) {
    for (int k = 0; k < 3; ++k) {
        GraphSlot &G = I.gslot[k];
        if (G.valid) {
            cudaGraphExecDestroy(G.exec);
            cudaGraphDestroy(G.graph);
            G.valid = 0;
        }
    }
}

// The coarse CTA takes the levels of at most `cap` cells (at most 1024: one
// per thread) whose subtree fits the shared-memory budget.
template <typename T> int Solver<T>::choose_cta(Instance &I, long long cap) {
    CLevels<T> P;
    const size_t budget = kCtaImageBytes;
    if (cap > kCtaCells) cap = kCtaCells;
    int lc0 = I.nlev - 1;
    while (lc0 > 0 && I.lev[lc0 - 1].g.ncell <= cap && Impl<T>::cta_levels(I, P, lc0 - 1) <= budget) --lc0;
    const size_t sm = Impl<T>::cta_levels(I, P, lc0);
    if (sm > budget) return OSCAR_E_INVALID_ARG;
    I.lc0 = lc0;
    I.cta_img_bytes = (sm + 15) & ~(size_t)15;
    I.cta_smem = I.cta_img_bytes;
    I.lg = -1;
    // the level above may join the CTA with its coefficients in global memory
    // when its x and b fit beside the image (never the finest level, whose x
    // and b are the Krylov vectors of the CG kernels)
    if (I.cta_global && lc0 - 1 >= 1 && I.lev[lc0 - 1].g.ncell <= kGlCells) {
        const size_t tot = Impl<T>::gl_bytes(I, lc0 - 1, I.cta_img_bytes);
        if (tot <= budget) {
            I.lg = lc0 - 1;
            I.cta_smem = tot;
        }
    }
    return 0;
}

template <typename T> int Solver<T>::setup(Instance &I, const uint8_t *solid_dev, const double *alpha0_dev) {
    BlockXScope bxs(I.block_x);
    GridD g = to_dev(I.g);
    L3 L = launch3(I.g);
    long long l0 = I.nlaunch;
    if (I.g.dim == 3) launchk(k_build_info<3>, L.grid, L.block, 0, I.stream, g, solid_dev, I.info, I.lev[0].fluid), ++I.nlaunch;
    else launchk(k_build_info<2>, L.grid, L.block, 0, I.stream, g, solid_dev, I.info, I.lev[0].fluid), ++I.nlaunch;
    launchk(k_load_alpha<T>, nblk(g.ncell), BS, 0, I.stream, g.ncell, I.info, alpha0_dev, (T *)I.alpha), ++I.nlaunch;
    for (int l = 1; l < I.nlev; ++l) {
        Level &F = I.lev[l - 1], &Lv = I.lev[l];
        L3 LC = launch3(Lv.g);
        launchk(k_mg_fluid_coarsen, LC.grid, LC.block, 0, I.stream, to_dev(F.g), to_dev(Lv.g), F.r[0], F.r[1], F.r[2],
                                                               F.fluid, Lv.fluid), ++I.nlaunch;
    }
    OSCAR_LAUNCH_CHECK();
    OSCAR_TRY(choose_cta(I, I.cta_cells));
    const size_t budget = kCtaImageBytes;
    // the attribute belongs to the kernel, not to this instance: it is set to
    // the budget (never lowered), so that instances of other sizes, created
    // while this one runs, cannot shrink it below what this one launches with
    cudaError_t e = I.g.dim == 3 ? cudaFuncSetAttribute(k_mg_coarse<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)budget)
                                 : cudaFuncSetAttribute(k_mg_coarse<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)budget);
    if (e == cudaSuccess)
        e = I.g.dim == 3 ? cudaFuncSetAttribute(k_mg_coarse_pack<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)budget)
                         : cudaFuncSetAttribute(k_mg_coarse_pack<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)budget);
    if (e != cudaSuccess) return OSCAR_E_CUDA;
    int rc = Impl<T>::interface_(I, I.alpha);
    I.nexec += I.nlaunch - l0;
    return rc;
}

template <typename T> int Solver<T>::drag_step(Instance &I, double dt) { return Impl<T>::run(I, 0, dt, 1); }

template <typename T> int Solver<T>::launch_step(Instance &I, int kind, double dt, int N) {
    int rc = Impl<T>::run_launch(I, kind, dt, N);
    if (rc) I.pending = -1;
    return rc;
}

template <typename T> int Solver<T>::finish_step(Instance &I, int *kf_out, double *test_out) {
    const int kind = I.pending, N = I.pending_N;
    int rc = Impl<T>::run_finish(I);
    if (rc == OSCAR_E_CUDA || rc == OSCAR_E_TIMEOUT) return rc;
    if (kind == 1) {
        I.last_kf = I.ctl_host[C_K];
        I.last_N = N;
        I.last_E = I.scal_host[S_E];
        I.last_dU = I.scal_host[S_DU];
    } else if (kind == 2) {
        I.last_E = I.scal_host[S_E];
        I.last_N = 1;
    }
    if (kf_out) *kf_out = kind == 1 ? I.ctl_host[C_K] : 1;
    if (test_out) *test_out = kind == 1 ? I.scal_host[S_TEST] : I.scal_host[S_E];
    return rc;
}

template <typename T> int Solver<T>::relax(Instance &I, double dt, int N, int *kf_out, double *test_out) {
    int rc = Impl<T>::run(I, 1, dt, N);
    if (rc == OSCAR_E_CUDA || rc == OSCAR_E_TIMEOUT) return rc;
    I.last_kf = I.ctl_host[C_K];
    I.last_N = N;
    I.last_E = I.scal_host[S_E];
    I.last_dU = I.scal_host[S_DU];
    if (kf_out) *kf_out = I.last_kf;
    if (test_out) *test_out = I.scal_host[S_TEST];
    return rc;
}

template <typename T> int Solver<T>::standard_step(Instance &I, double dt) {
    int rc = Impl<T>::run(I, 2, dt, 1);
    if (rc == OSCAR_E_CUDA || rc == OSCAR_E_TIMEOUT) return rc;
    I.last_E = I.scal_host[S_E];
    I.last_N = 1;
    return rc;
}

template <typename T>
__global__ void k_report_u(int n, const T *__restrict__ uvd, const double *__restrict__ usum, double invN,
                           double *__restrict__ out) {
    griddep_wait();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = (double)uvd[c] + usum[c] * invN;
}
static __global__ void k_add_pd(int n, const double *__restrict__ a, const double *__restrict__ b,
                                double *__restrict__ out) {
    griddep_wait();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = a[c] + b[c];
}

template <typename T> int Solver<T>::field_to_device(Instance &I, int which, double *dst, size_t n) {
    BlockXScope bxs(I.block_x);
    int nc = I.g.ncell;
    cudaStream_t s = I.stream;
    auto cvt = [&](const void *src, size_t len) {
        launchk(k_convert<T, double>, nblk(len), BS, 0, s, (int)len, (const T *)src, dst), ++I.nlaunch, ++I.nexec;
    };
    if (which == OSCAR_FIELD_ALPHA) cvt(I.alpha, nc);
    else if (which == OSCAR_FIELD_P) launchk(k_add_pd, nblk(nc), BS, 0, s, nc, I.p_vd, I.p_cr, dst), ++I.nlaunch, ++I.nexec;
    else if (which >= 2 && which <= 4) {
        int a = which - 2;
        if (a >= I.g.dim) cudaMemsetAsync(dst, 0, n * sizeof(double), s);
        else launchk(k_report_u<T>, nblk(nc), BS, 0, s, nc, (const T *)I.u_vd[a], I.u_sum[a], 1.0 / (double)I.last_N, dst),
                 ++I.nlaunch, ++I.nexec;
    } else if (which >= 5 && which <= 10) {
        int a = (which - 5) % 3;
        void *const *src = which < 8 ? I.u_vd : I.u_cr;
        if (a >= I.g.dim) cudaMemsetAsync(dst, 0, n * sizeof(double), s);
        else cvt(src[a], nc);
    } else if (which == OSCAR_FIELD_P_VD) cudaMemcpyAsync(dst, I.p_vd, nc * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else if (which == OSCAR_FIELD_P_CR) cudaMemcpyAsync(dst, I.p_cr, nc * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else if (which == OSCAR_FIELD_KAPPA) cvt(I.kappa, nc);
    else if (which >= 14 && which <= 22) {
        int a = (which - 14) % 3;
        void *const *src = which < 17 ? I.phi_vd : (which < 20 ? I.phi_cr : I.nf);
        if (a >= I.g.dim) cudaMemsetAsync(dst, 0, n * sizeof(double), s);
        else cvt(src[a], I.g.nf[a]);
    } else return OSCAR_E_INVALID_ARG;
    OSCAR_LAUNCH_CHECK();
    return 0;
}

template <typename T> int Solver<T>::field_from_device(Instance &I, int which, const double *src, size_t n) {
    BlockXScope bxs(I.block_x);
    int nc = I.g.ncell;
    cudaStream_t s = I.stream;
    auto cvt = [&](void *dst, size_t len) {
        launchk(k_convert<double, T>, nblk(len), BS, 0, s, (int)len, src, (T *)dst), ++I.nlaunch, ++I.nexec;
    };
    if (which == OSCAR_FIELD_ALPHA) {
        launchk(k_load_alpha<T>, nblk(nc), BS, 0, s, nc, I.info, src, (T *)I.alpha), ++I.nlaunch, ++I.nexec;
        OSCAR_LAUNCH_CHECK();
        long long l0 = I.nlaunch;
        int rc = Impl<T>::interface_(I, I.alpha);
        I.nexec += I.nlaunch - l0;
        return rc;
    } else if (which >= 5 && which <= 10) {
        int a = (which - 5) % 3;
        if (a >= I.g.dim) return OSCAR_E_INVALID_ARG;
        cvt(which < 8 ? I.u_vd[a] : I.u_cr[a], nc);
    } else if (which == OSCAR_FIELD_P_VD || which == OSCAR_FIELD_P) {
        cudaMemcpyAsync(I.p_vd, src, nc * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else if (which == OSCAR_FIELD_P_CR) {
        cudaMemcpyAsync(I.p_cr, src, nc * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else if (which >= 14 && which <= 19) {
        int a = (which - 14) % 3;
        if (a >= I.g.dim) return OSCAR_E_INVALID_ARG;
        cvt(which < 17 ? I.phi_vd[a] : I.phi_cr[a], I.g.nf[a]);
    } else return OSCAR_E_INVALID_ARG;
    OSCAR_LAUNCH_CHECK();
    return 0;
}

template <typename T> int Solver<T>::phase_volume(Instance &I, double *out) {
    BlockXScope bxs(I.block_x);
    launchk(k_sum_to<T>, kRedBlocks, BS, 0, I.stream, I.g.ncell, (const T *)I.alpha, I.g.V, I.partials, I.ticket, I.scal,
                                                 S_VOL), ++I.nlaunch, ++I.nexec;
    OSCAR_LAUNCH_CHECK();
    if (cudaMemcpyAsync(I.scal_host, I.scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, I.stream) != cudaSuccess)
        return OSCAR_E_CUDA;
    int rc = sync_bounded(I.stream, kSyncTimeoutSec);
    if (rc) return rc;
    *out = I.scal_host[S_VOL];
    return 0;
}

}  // namespace oscar
