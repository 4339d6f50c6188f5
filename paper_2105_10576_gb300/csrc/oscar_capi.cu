// C ABI of the OSCAR library (declared in include/oscar.h): instance
// creation, memory layout, multigrid hierarchy and dispatch to the FP64 or
// mixed-precision solver.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cxxabi.h>

#include <chrono>
#include <new>
#include <string>
#include <vector>

#include "oscar_internal.h"

struct oscar_instance {
    oscar::Instance I;
};

namespace oscar {

int sync_bounded(cudaStream_t s, double timeout_sec) {
    auto t0 = std::chrono::steady_clock::now();
    for (unsigned long it = 0;; ++it) {
        cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) return 0;
        if (e != cudaErrorNotReady) {
            fprintf(stderr, "oscar: stream error %s\n", cudaGetErrorString(e));
            return OSCAR_E_CUDA;
        }
        if ((it & 1023) == 0) {
            double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_sec) return OSCAR_E_TIMEOUT;
        }
    }
}

// accumulate the recorded event pairs into their entries (waits for st)
int prof_drain(Profiler *P, cudaStream_t st) {
    if (P->n == 0) return 0;
    int rc = sync_bounded(st, kSyncTimeoutSec);
    for (int s = 0; s < P->n; ++s) {
        float ms = 0.f;
        if (!rc && cudaEventElapsedTime(&ms, P->ev0[s], P->ev1[s]) == cudaSuccess) {
            P->ent[P->slot_entry[s]].total_ms += ms;
            P->ent[P->slot_entry[s]].launches += 1;
        } else {
            cudaGetLastError();
            P->dropped++;
        }
    }
    P->n = 0;
    return rc;
}

int prof_begin(Profiler *P, cudaStream_t st, const void *fn, dim3 grid, dim3 block) {
    const unsigned gsz = grid.x * grid.y * grid.z, bsz = block.x * block.y * block.z;
    int e = 0;
    while (e < P->nent && !(P->ent[e].fn == fn && P->ent[e].grid == gsz && P->ent[e].block == bsz)) ++e;
    if (e == P->nent) {
        if (P->nent >= kProfKinds) { P->dropped++; return -1; }
        P->ent[e].fn = fn;
        P->ent[e].grid = gsz;
        P->ent[e].block = bsz;
        P->ent[e].total_ms = 0.0;
        P->ent[e].launches = 0;
        P->nent++;
    }
    if (P->n >= kProfPool && prof_drain(P, st)) { P->dropped++; return -1; }
    int s = P->n++;
    P->slot_entry[s] = e;
    cudaEventRecord(P->ev0[s], st);
    return s;
}

void prof_end(Profiler *P, cudaStream_t st, int slot) {
    if (slot >= 0) cudaEventRecord(P->ev1[slot], st);
}

size_t field_len(const Instance &I, int which) {
    if (which >= 0 && which <= OSCAR_FIELD_KAPPA) return (size_t)I.g.ncell;
    if (which >= OSCAR_FIELD_PHI_VD && which <= OSCAR_FIELD_NF + 2) return (size_t)I.g.nf[(which - OSCAR_FIELD_PHI_VD) % 3];
    return 0;
}

static GridH make_grid(int dim, int nx, int ny, int nz, double hx, double hy, double hz) {
    GridH g;
    g.dim = dim;
    g.nx = nx; g.ny = ny; g.nz = dim == 3 ? nz : 1;
    g.ncell = g.nx * g.ny * g.nz;
    g.nf[0] = (g.nx + 1) * g.ny * g.nz;
    g.nf[1] = g.nx * (g.ny + 1) * g.nz;
    g.nf[2] = g.nx * g.ny * (g.nz + 1);
    g.h[0] = hx; g.h[1] = hy; g.h[2] = hz;
    g.V = 1.0;
    for (int a = 0; a < dim; ++a) g.V *= g.h[a];
    for (int a = 0; a < 3; ++a) g.S[a] = a < dim ? g.V / g.h[a] : 0.0;
    return g;
}

// Coarsening: halve every direction whose spacing is below twice the smallest
// spacing (semi-coarsening of the strongly coupled directions on anisotropic
// cells), until at most 64 cells remain.
static void build_hierarchy(Instance &I) {
    I.nlev = 1;
    I.lev[0].g = I.g;
    while (I.nlev < kMaxLevels) {
        GridH &g = I.lev[I.nlev - 1].g;
        int *r = I.lev[I.nlev - 1].r;
        r[0] = r[1] = r[2] = 1;
        if (g.ncell <= 8) break;
        int n[3] = {g.nx, g.ny, g.nz};
        double hmin = 1e300;
        for (int a = 0; a < g.dim; ++a)
            if (n[a] > 1 && g.h[a] < hmin) hmin = g.h[a];
        bool any = false;
        for (int a = 0; a < g.dim; ++a)
            if (n[a] > 1 && g.h[a] < 2.0 * hmin) { r[a] = 2; any = true; }
        if (!any) break;
        GridH c = make_grid(g.dim, (g.nx + r[0] - 1) / r[0], (g.ny + r[1] - 1) / r[1], (g.nz + r[2] - 1) / r[2],
                            g.h[0] * r[0], g.h[1] * r[1], g.h[2] * r[2]);
        I.lev[I.nlev].g = c;
        I.lev[I.nlev].r[0] = I.lev[I.nlev].r[1] = I.lev[I.nlev].r[2] = 1;
        ++I.nlev;
    }
}

struct Carver {
    char *base;
    size_t off;
    bool dry;
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = dry ? nullptr : base + off;
        off += bytes;
        return p;
    }
};

static void carve(Instance &I, Carver &C) {
    size_t es = I.prec == OSCAR_FP64 ? sizeof(double) : sizeof(float);
    size_t nc = I.g.ncell;
    I.info = (uint32_t *)C.take(nc * sizeof(uint32_t));
    void **cells[] = {&I.alpha, &I.alpha_new, &I.alpha_s, &I.alpha_tmp, &I.kappa, &I.aL, &I.Pp, &I.Pm, &I.Rp, &I.Rm, &I.rA};
    for (void **p : cells) *p = C.take(nc * es);
    for (int a = 0; a < 3; ++a) {
        I.hbya[a] = C.take(nc * es);
        I.vold[a] = C.take(nc * es);
        I.u_vd[a] = C.take(nc * es);
        I.u_cr[a] = C.take(nc * es);
        I.u_sum[a] = (double *)C.take(nc * sizeof(double));
    }
    for (int q = 0; q < 9; ++q) I.G[q] = C.take(nc * es);
    I.p_vd = (double *)C.take(nc * sizeof(double));
    I.p_cr = (double *)C.take(nc * sizeof(double));
    I.cg_b = (double *)C.take(nc * sizeof(double));
    I.cg_r = (double *)C.take(nc * sizeof(double));
    I.cg_z = (double *)C.take(nc * sizeof(double));
    I.cg_p = (double *)C.take(nc * sizeof(double));
    I.cg_Ap = (double *)C.take(nc * sizeof(double));
    I.cg_e = C.take(nc * es);
    I.cg_r64 = I.prec != OSCAR_FP64 ? (double *)C.take(nc * sizeof(double)) : nullptr;
    if (I.prec != OSCAR_FP64) {
        for (int a = 0; a < 3; ++a) I.cf64[a] = (double *)C.take((size_t)I.g.nf[a] * sizeof(double));
    }
    for (int a = 0; a < 3; ++a) {
        size_t nf = I.g.nf[a];
        I.nf[a] = C.take(nf * es);
        I.phi_vd[a] = C.take(nf * es);
        I.phi_cr[a] = C.take(nf * es);
        I.phic[a] = C.take(nf * es);
        I.phis[a] = C.take(nf * es);
        I.fst[a] = C.take(nf * es);
    }
    for (int l = 0; l < I.nlev; ++l) {
        Level &L = I.lev[l];
        size_t n = L.g.ncell;
        L.fluid = (uint8_t *)C.take(n);
        for (int a = 0; a < 3; ++a) L.c[a] = C.take((size_t)L.g.nf[a] * es);
        L.diag = C.take(n * es);
        L.idiag = C.take(n * es);
        if (l == 0 && I.prec == OSCAR_FP64) {
            for (int a = 0; a < 3; ++a) I.cf64[a] = (double *)L.c[a];
        }
        L.x = C.take(n * es);
        L.b = C.take(n * es);
        L.res = C.take(n * es);
    }
    I.stage_dev = (double *)C.take(I.stage_len * sizeof(double));
    I.cta_img = C.take(kCtaImageBytes);
    I.partials = (double *)C.take((size_t)kRedSlots * I.red_stride * sizeof(double));
    I.scal = (double *)C.take(S_COUNT * sizeof(double));
    I.ctl = (int *)C.take(C_COUNT * sizeof(int));
    I.ticket = (unsigned *)C.take(sizeof(unsigned));
}

// Partial-sum slots per reduction: the fixed reduction grid, or the blocks
// of the largest cell launch over every block shape a schedule may select
// (block_x 32 .. 256; the half-width launches of the red-black sweeps are
// covered by the full-width count).
static int reduction_stride(const GridH &g) {
    long long nb = kRedBlocks;
    for (int bx = 32; bx <= 256; bx *= 2) {
        const int by = 256 / bx;
        const long long b = (long long)((g.nx + bx - 1) / bx) * ((g.ny + by - 1) / by) * g.nz;
        if (b > nb) nb = b;
    }
    return (int)nb;
}

static int validate(const oscar_params *p) {
    if (!p) return OSCAR_E_INVALID_ARG;
    if (p->dim != 2 && p->dim != 3) return OSCAR_E_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || (p->dim == 3 && p->nz < 1)) return OSCAR_E_INVALID_ARG;
    double ncell = (double)p->nx * p->ny * (p->dim == 3 ? p->nz : 1);
    double nface = (double)(p->nx + 1) * p->ny * (p->dim == 3 ? p->nz + 1 : 1) * 2.0;
    if (ncell > 2.0e9 || nface > 2.0e9) return OSCAR_E_INVALID_ARG;
    if (!(p->hx > 0) || !(p->hy > 0) || (p->dim == 3 && !(p->hz > 0))) return OSCAR_E_INVALID_ARG;
    if (!(p->rho1 > 0) || !(p->rho2 > 0) || p->mu1 < 0 || p->mu2 < 0 || p->sigma < 0) return OSCAR_E_INVALID_ARG;
    if (p->n_piso < 1 || p->n_smooth < 0 || p->cg_maxit < 1 || !(p->cg_rtol > 0)) return OSCAR_E_INVALID_ARG;
    if (p->precision != OSCAR_FP64 && p->precision != OSCAR_MIXED) return OSCAR_E_INVALID_ARG;
    if (p->conv_mode != OSCAR_CONV_PRES_RESID && p->conv_mode != OSCAR_CONV_DU_MAX && p->conv_mode != OSCAR_CONV_AREA)
        return OSCAR_E_INVALID_ARG;
    return 0;
}

}  // namespace oscar

using namespace oscar;

extern "C" {

int oscar_timesteps(const oscar_params *p, const uint8_t *solid, double c_cfl, double out[4]) {
    if (!p || !out || !(p->U_inlet > 0) || !(p->sigma > 0) || !(c_cfl > 0)) return OSCAR_E_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || (p->dim == 3 && p->nz < 1)) return OSCAR_E_INVALID_ARG;
    double hmin = p->hx;
    if (p->hy < hmin) hmin = p->hy;
    if (p->dim == 3 && p->hz < hmin) hmin = p->hz;
    // CFL velocity: the injected flux U A(inlet) crosses every x-section, so
    // the largest section-mean speed is U A(inlet) / min_x A(x)
    double u_cfl = p->U_inlet;
    if (solid) {
        const long long nyz = (long long)p->ny * (p->dim == 3 ? p->nz : 1);
        std::vector<long long> area(p->nx, 0);
        for (long long r = 0; r < nyz; ++r) {
            const uint8_t *row = solid + r * p->nx;
            for (int i = 0; i < p->nx; ++i) area[i] += row[i] == 0;
        }
        long long amin = area[0];
        for (int i = 1; i < p->nx; ++i) amin = area[i] < amin ? area[i] : amin;
        if (area[0] > 0) {
            if (amin == 0) return OSCAR_E_INVALID_ARG;   // the inlet does not reach the outlet
            u_cfl = p->U_inlet * (double)area[0] / (double)amin;
        }
    }
    double dt_cfl = p->hx / u_cfl;
    double rho_bar = 0.5 * (p->rho1 + p->rho2);
    double dt_b = sqrt(rho_bar * hmin * hmin * hmin / (2.0 * M_PI * p->sigma));
    double dt_vd = c_cfl * dt_cfl;
    out[0] = dt_cfl;
    out[1] = dt_b;
    out[2] = dt_vd;
    out[3] = floor(dt_vd / dt_b) + 1.0;
    return 0;
}

const char *oscar_strerror(int code) {
    switch (code) {
        case OSCAR_OK: return "ok";
        case OSCAR_E_INVALID_ARG: return "invalid argument";
        case OSCAR_E_OOM: return "out of device memory";
        case OSCAR_E_NOT_CONVERGED: return "pressure solve hit its iteration cap";
        case OSCAR_E_NAN: return "non-finite value in the solution";
        case OSCAR_E_TIMEOUT: return "bounded wait for the stream timed out";
        case OSCAR_E_CUDA: return "CUDA error";
        default: return "unknown error";
    }
}

// grid, multigrid hierarchy and arena layout of an instance (no allocation)
static void plan(Instance &I, const oscar_params *p) {
    I.P = *p;
    I.prec = p->precision;
    I.g = make_grid(p->dim, p->nx, p->ny, p->nz, p->hx, p->hy, p->hz);
    build_hierarchy(I);
    I.red_stride = reduction_stride(I.g);
    size_t stage = I.g.ncell;
    for (int a = 0; a < 3; ++a) if ((size_t)I.g.nf[a] > stage) stage = I.g.nf[a];
    I.stage_len = stage;
    Carver dry{nullptr, 0, true};
    carve(I, dry);
    I.arena_bytes = dry.off + 256;
}

int oscar_footprint(const oscar_params *p, size_t *bytes_out) {
    if (!bytes_out) return OSCAR_E_INVALID_ARG;
    int rc = validate(p);
    if (rc) return rc;
    Instance *I = new (std::nothrow) Instance();
    if (!I) return OSCAR_E_OOM;
    memset(I, 0, sizeof(Instance));
    plan(*I, p);
    *bytes_out = I->arena_bytes;
    delete I;
    return 0;
}

int oscar_create(const oscar_params *p, const uint8_t *solid, const double *alpha0, void *stream,
                 oscar_handle *out) {
    if (!out) return OSCAR_E_INVALID_ARG;
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    if (!solid || !alpha0) return OSCAR_E_INVALID_ARG;
    oscar_instance *H = new (std::nothrow) oscar_instance();
    if (!H) return OSCAR_E_OOM;
    Instance &I = H->I;
    memset(&I, 0, sizeof(Instance));
    I.P = *p;
    I.prec = p->precision;
    I.stream = (cudaStream_t)stream;
    if (!I.stream) {   // graphs cannot be captured on the legacy default stream: use a private one
        if (cudaStreamCreateWithFlags(&I.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete H;
            return OSCAR_E_CUDA;
        }
        I.own_stream = 1;
    }
    {
        const char *e = getenv("OSCAR_EAGER");
        I.eager = (e && e[0] == '1') ? 1 : 0;
    }
    I.g = make_grid(p->dim, p->nx, p->ny, p->nz, p->hx, p->hy, p->hz);
    I.cos_theta = cos(p->theta_deg * M_PI / 180.0);
    I.deltaN = 1e-8 / pow(I.g.V, 1.0 / p->dim);
    I.last_N = 1;
    I.pending = -1;
    I.mg_nu = 2;
    I.mg_nu_c = 2;
    I.mg_coarse_sweeps = 4;
    I.mg_nu_cta = 2;
    I.coarse_refresh = 8;
    I.cta_cells = 1024;
    I.block_x = 0;
    I.cta_global = 1;
    I.repeat_fine = 0;
    I.lg = -1;
    long long nf = 0;
    for (int c = 0; c < I.g.ncell; ++c) nf += solid[c] == 0;
    I.n_fluid = nf;
    if (nf == 0) { delete H; return OSCAR_E_INVALID_ARG; }
    build_hierarchy(I);
    I.red_stride = reduction_stride(I.g);
    I.lc0 = I.nlev - 1;   // refined by the solver set-up (shared-memory budget of the coarse CTA)
    size_t stage = I.g.ncell;
    for (int a = 0; a < 3; ++a) if ((size_t)I.g.nf[a] > stage) stage = I.g.nf[a];
    I.stage_len = stage;
    Carver dry{nullptr, 0, true};
    carve(I, dry);
    I.arena_bytes = dry.off + 256;
    if (cudaMalloc(&I.arena, I.arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete H;
        return OSCAR_E_OOM;
    }
    Carver wet{(char *)I.arena, 0, false};
    carve(I, wet);
    bool streams_ok = true;
    for (int q = 0; q < 4; ++q)
        if (cudaStreamCreateWithFlags(&I.side[q], cudaStreamNonBlocking) != cudaSuccess) streams_ok = false;
    if (!streams_ok || cudaMallocHost(&I.scal_host, S_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&I.ctl_host, C_COUNT * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&I.stage_host, stage * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(I.arena);
        delete H;
        return OSCAR_E_OOM;
    }
    if (cudaMemsetAsync(I.arena, 0, I.arena_bytes, I.stream) != cudaSuccess) { oscar_destroy(H); return OSCAR_E_CUDA; }
    // upload the mask and alpha0 through a temporary device buffer
    void *tmp = nullptr;
    size_t tbytes = (size_t)I.g.ncell * (sizeof(double) + 1);
    if (cudaMalloc(&tmp, tbytes) != cudaSuccess) { cudaGetLastError(); oscar_destroy(H); return OSCAR_E_OOM; }
    double *a0d = (double *)tmp;
    uint8_t *sd = (uint8_t *)(a0d + I.g.ncell);
    cudaMemcpyAsync(a0d, alpha0, (size_t)I.g.ncell * sizeof(double), cudaMemcpyHostToDevice, I.stream);
    cudaMemcpyAsync(sd, solid, (size_t)I.g.ncell, cudaMemcpyHostToDevice, I.stream);
    rc = I.prec == OSCAR_FP64 ? Solver<double>::setup(I, sd, a0d) : Solver<float>::setup(I, sd, a0d);
    int rc2 = sync_bounded(I.stream, kSyncTimeoutSec);
    cudaFree(tmp);
    if (rc || rc2) { oscar_destroy(H); return rc ? rc : rc2; }
    *out = H;
    return 0;
}

int oscar_destroy(oscar_handle h) {
    if (!h) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.arena) {
        sync_bounded(I.stream, kSyncTimeoutSec);
        if (I.prec == OSCAR_FP64) Solver<double>::release_graphs(I);
        else Solver<float>::release_graphs(I);
        cudaFree(I.arena);
    }
    for (int q = 0; q < 4; ++q)
        if (I.side[q]) cudaStreamDestroy(I.side[q]);
    if (I.own_stream && I.stream) cudaStreamDestroy(I.stream);
    if (I.ctl_host) cudaFreeHost(I.ctl_host);
    if (I.prof) {
        if (I.prof->created)
            for (int s = 0; s < kProfPool; ++s) { cudaEventDestroy(I.prof->ev0[s]); cudaEventDestroy(I.prof->ev1[s]); }
        delete I.prof;
    }
    if (I.scal_host) cudaFreeHost(I.scal_host);
    if (I.stage_host) cudaFreeHost(I.stage_host);
    delete h;
    return 0;
}

int oscar_drag_step_async(oscar_handle h, double dt_vd) {
    if (!h || !(dt_vd > 0)) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;
    return I.prec == OSCAR_FP64 ? Solver<double>::launch_step(I, 0, dt_vd, 1) : Solver<float>::launch_step(I, 0, dt_vd, 1);
}

int oscar_relax_async(oscar_handle h, double dt_cr, int N) {
    if (!h || !(dt_cr > 0) || N < 1) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;
    if (I.P.conv_mode == OSCAR_CONV_DU_MAX && !(I.P.U_inlet > 0)) return OSCAR_E_INVALID_ARG;
    return I.prec == OSCAR_FP64 ? Solver<double>::launch_step(I, 1, dt_cr, N) : Solver<float>::launch_step(I, 1, dt_cr, N);
}

int oscar_standard_step_async(oscar_handle h, double dt) {
    if (!h || !(dt > 0)) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;
    return I.prec == OSCAR_FP64 ? Solver<double>::launch_step(I, 2, dt, 1) : Solver<float>::launch_step(I, 2, dt, 1);
}

int oscar_query(oscar_handle h) {
    if (!h) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending < 0) return OSCAR_E_INVALID_ARG;
    cudaError_t e = cudaStreamQuery(I.stream);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    cudaGetLastError();
    return OSCAR_E_CUDA;
}

int oscar_wait(oscar_handle h, int *k_f_out, double *test_out) {
    if (!h) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending < 0) return OSCAR_E_INVALID_ARG;
    return I.prec == OSCAR_FP64 ? Solver<double>::finish_step(I, k_f_out, test_out)
                                : Solver<float>::finish_step(I, k_f_out, test_out);
}

int oscar_drag_step(oscar_handle h, double dt_vd) {
    if (!h || !(dt_vd > 0)) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    return I.prec == OSCAR_FP64 ? Solver<double>::drag_step(I, dt_vd) : Solver<float>::drag_step(I, dt_vd);
}

int oscar_relax(oscar_handle h, double dt_cr, int N, int *k_f_out, double *test_out) {
    if (!h || !(dt_cr > 0) || N < 1) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    if (I.P.conv_mode == OSCAR_CONV_DU_MAX && !(I.P.U_inlet > 0)) return OSCAR_E_INVALID_ARG;
    return I.prec == OSCAR_FP64 ? Solver<double>::relax(I, dt_cr, N, k_f_out, test_out)
                                : Solver<float>::relax(I, dt_cr, N, k_f_out, test_out);
}

int oscar_standard_step(oscar_handle h, double dt) {
    if (!h || !(dt > 0)) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    return I.prec == OSCAR_FP64 ? Solver<double>::standard_step(I, dt) : Solver<float>::standard_step(I, dt);
}

int oscar_fields_device(oscar_handle h, int which, double *dev_out, size_t n) {
    if (!h || !dev_out) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    size_t len = field_len(I, which);
    if (len == 0 || n != len) return OSCAR_E_INVALID_ARG;
    return I.prec == OSCAR_FP64 ? Solver<double>::field_to_device(I, which, dev_out, n)
                                : Solver<float>::field_to_device(I, which, dev_out, n);
}

int oscar_fields(oscar_handle h, int which, double *host_out, size_t n) {
    if (!h || !host_out) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    size_t len = field_len(I, which);
    if (len == 0 || n != len) return OSCAR_E_INVALID_ARG;
    int rc = I.prec == OSCAR_FP64 ? Solver<double>::field_to_device(I, which, I.stage_dev, len)
                                  : Solver<float>::field_to_device(I, which, I.stage_dev, len);
    if (!rc && cudaMemcpyAsync(I.stage_host, I.stage_dev, len * sizeof(double), cudaMemcpyDeviceToHost, I.stream) !=
                   cudaSuccess)
        rc = OSCAR_E_CUDA;
    int rc2 = sync_bounded(I.stream, kSyncTimeoutSec);
    if (rc) return rc;
    if (rc2) return rc2;
    memcpy(host_out, I.stage_host, len * sizeof(double));
    return 0;
}

int oscar_set_field(oscar_handle h, int which, const double *host_in, size_t n) {
    if (!h || !host_in) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    size_t len = field_len(I, which);
    if (len == 0 || n != len) return OSCAR_E_INVALID_ARG;
    int rc = sync_bounded(I.stream, kSyncTimeoutSec);
    if (rc) return rc;
    memcpy(I.stage_host, host_in, len * sizeof(double));
    if (cudaMemcpyAsync(I.stage_dev, I.stage_host, len * sizeof(double), cudaMemcpyHostToDevice, I.stream) !=
        cudaSuccess)
        return OSCAR_E_CUDA;
    rc = I.prec == OSCAR_FP64 ? Solver<double>::field_from_device(I, which, I.stage_dev, len)
                              : Solver<float>::field_from_device(I, which, I.stage_dev, len);
    int rc2 = sync_bounded(I.stream, kSyncTimeoutSec);
    return rc ? rc : rc2;
}

int oscar_get_schedule(oscar_handle h, oscar_schedule *out) {
    if (!h || !out) return OSCAR_E_INVALID_ARG;
    const Instance &I = h->I;
    out->mg_nu = I.mg_nu;
    out->mg_nu_mid = I.mg_nu_c;
    out->mg_nu_cta = I.mg_nu_cta;
    out->cta_cells = I.cta_cells;
    out->coarse_refresh = I.coarse_refresh;
    out->block_x = I.block_x;
    out->cta_global = I.cta_global;
    return 0;
}

int oscar_set_schedule(oscar_handle h, const oscar_schedule *s) {
    if (!h || !s) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    if (s->mg_nu < 1 || s->mg_nu > 4 || s->mg_nu_mid < 1 || s->mg_nu_mid > 4 || s->mg_nu_cta < 1 ||
        s->mg_nu_cta > 6 || s->cta_cells < 1 || s->cta_cells > 1024 || s->coarse_refresh < 1 ||
        s->coarse_refresh > 1000)
        return OSCAR_E_INVALID_ARG;
    if (!(s->block_x == 0 || s->block_x == 32 || s->block_x == 64 || s->block_x == 128 || s->block_x == 256))
        return OSCAR_E_INVALID_ARG;
    if (s->cta_global != 0 && s->cta_global != 1) return OSCAR_E_INVALID_ARG;
    int rc = sync_bounded(I.stream, kSyncTimeoutSec);
    if (rc) return rc;
    const int lc0 = I.lc0, lg = I.lg, cg = I.cta_global;
    const size_t sm = I.cta_smem, ib = I.cta_img_bytes;
    I.cta_global = s->cta_global;
    rc = I.prec == OSCAR_FP64 ? Solver<double>::choose_cta(I, s->cta_cells) : Solver<float>::choose_cta(I, s->cta_cells);
    if (rc) {   // keep the previous schedule
        I.lc0 = lc0;
        I.lg = lg;
        I.cta_global = cg;
        I.cta_smem = sm;
        I.cta_img_bytes = ib;
        return rc;
    }
    I.mg_nu = s->mg_nu;
    I.mg_nu_c = s->mg_nu_mid;
    I.mg_nu_cta = s->mg_nu_cta;
    I.cta_cells = s->cta_cells;
    I.coarse_refresh = s->coarse_refresh;
    I.block_x = s->block_x;
    if (I.prec == OSCAR_FP64) Solver<double>::release_graphs(I);
    else Solver<float>::release_graphs(I);
    return 0;
}

int oscar_stats(oscar_handle h, oscar_stats_t *out) {
    if (!h || !out) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    double vol = 0.0;
    int rc = I.prec == OSCAR_FP64 ? Solver<double>::phase_volume(I, &vol) : Solver<float>::phase_volume(I, &vol);
    if (rc) return rc;
    out->k_f = I.last_kf;
    out->N = I.last_N;
    out->E_last = I.last_E;
    out->dU_last = I.last_dU;
    out->cg_iters_total = I.cg_iters_total;
    out->cg_iters_last = I.cg_iters_last;
    out->mg_levels = I.nlev;
    out->phase_volume = vol;
    out->n_fluid = I.n_fluid;
    out->cell_updates = I.cell_updates;
    out->device_bytes = I.arena_bytes;
    out->kernel_launches = I.nexec;
    out->mg_first_cta_level = I.lc0;
    out->mg_cta_global_level = I.lg;
    return 0;
}

}  // extern "C"

extern "C" {

int oscar_profile_repeat(oscar_handle h, int enable) {
    if (!h) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    int rc = sync_bounded(I.stream, kSyncTimeoutSec);
    if (rc) return rc;
    const int v = enable ? 1 : 0;
    if (v != I.repeat_fine) {   // the launch sequence changes: graphs are captured again
        I.repeat_fine = v;
        if (I.prec == OSCAR_FP64) Solver<double>::release_graphs(I);
        else Solver<float>::release_graphs(I);
    }
    return 0;
}

int oscar_profile(oscar_handle h, int enable) {
    if (!h) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    if (!I.prof) {
        I.prof = new (std::nothrow) Profiler();
        if (!I.prof) return OSCAR_E_OOM;
        memset(I.prof, 0, sizeof(Profiler));
    }
    Profiler *P = I.prof;
    if (enable && !P->created) {
        for (int s = 0; s < kProfPool; ++s) {
            if (cudaEventCreate(&P->ev0[s]) != cudaSuccess || cudaEventCreate(&P->ev1[s]) != cudaSuccess) {
                cudaGetLastError();
                for (int q = 0; q <= s; ++q) { cudaEventDestroy(P->ev0[q]); cudaEventDestroy(P->ev1[q]); }
                return OSCAR_E_CUDA;
            }
        }
        P->created = 1;
    }
    if (enable) {   // a new recording: clear the previous one
        P->n = 0;
        P->nent = 0;
        P->dropped = 0;
    } else if (P->created) {
        int rc = prof_drain(P, I.stream);
        if (rc) return rc;
    }
    P->enabled = enable ? 1 : 0;
    return 0;
}

int oscar_profile_read(oscar_handle h, int index, int *count_out, char *name_out, size_t name_cap,
                       unsigned *grid_out, double *total_ms, long long *launches) {
    if (!h || index < 0) return OSCAR_E_INVALID_ARG;
    Instance &I = h->I;
    if (I.pending >= 0) return OSCAR_E_INVALID_ARG;   // a launched step awaits oscar_wait
    Profiler *P = I.prof;
    const int n = P ? P->nent : 0;
    if (count_out) *count_out = n;
    if (P && P->created) {
        int rc = prof_drain(P, I.stream);
        if (rc) return rc;
    }
    if (index >= n) return OSCAR_E_INVALID_ARG;
    const ProfEntry &E = P->ent[index];
    if (name_out && name_cap > 0) {
        const char *nm = nullptr;
        if (cudaFuncGetName(&nm, E.fn) != cudaSuccess || !nm) {
            cudaGetLastError();
            nm = "?";
        }
        // readable form: "k_name<template args>" without the namespace and parameters
        std::string out = nm;
        int st = 0;
        char *dm = abi::__cxa_demangle(nm, nullptr, nullptr, &st);
        if (st == 0 && dm) {
            out = dm;
            free(dm);
            size_t lt = out.find('<'), lp = out.find('(');
            size_t cut = lp;
            if (lt != std::string::npos && lt < lp) {   // the parameter list follows the matching '>'
                int depth = 0;
                for (size_t q = lt; q < out.size(); ++q) {
                    if (out[q] == '<') ++depth;
                    else if (out[q] == '>' && --depth == 0) { cut = q + 1; break; }
                }
            }
            if (cut != std::string::npos) out = out.substr(0, cut);
            if (out.rfind("void ", 0) == 0) out = out.substr(5);
            for (size_t q; (q = out.find("oscar::")) != std::string::npos;) out.erase(q, 7);
        }
        snprintf(name_out, name_cap, "%s", out.c_str());
    }
    if (grid_out) *grid_out = E.grid;
    if (total_ms) *total_ms = E.total_ms;
    if (launches) *launches = E.launches;
    return 0;
}

}  // extern "C"
