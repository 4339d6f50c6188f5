// OSCAR hot path on sm_103a: stencil, transport, interface, PISO and MG-PCG
// kernels plus the per-precision orchestration of the drag step, the
// capillary-relaxation loop and standard stepping (Maes & Menke, arXiv
// 2105.10576, Sections 2-3).
//
// Every kernel is memory bound (no dense contraction anywhere), so there are
// no tensor-core paths. Layout: structure-of-arrays cell fields (x fastest) and
// one face array per direction; one thread per cell (or per face) with
// coalesced x-sweeps; all reductions run on a fixed grid of kRedBlocks blocks
// and finish in one block, so every sum is deterministic run to run.
//
// Included by exactly one translation unit per element type T (double: the
// FP64 path; float: the mixed path whose CG vectors, dots, norms and
// accumulators stay in double).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <utility>

#include "oscar_internal.h"

namespace oscar {

enum : int { FT_NONE = 0, FT_INTERIOR = 1, FT_WALL = 2, FT_INLET = 3, FT_OUTLET = 4 };
constexpr uint32_t INFO_FLUID = 1u << 31;
constexpr int BS = 256;

__device__ __forceinline__ int ftype(uint32_t info, int a, int s) { return (info >> (3 * (2 * a + s))) & 7; }

struct GridD {
    int nx, ny, nz, ncell;
    double h[3], S[3], V;
};

inline GridD to_dev(const GridH &g) {
    GridD d;
    d.nx = g.nx; d.ny = g.ny; d.nz = g.nz; d.ncell = g.ncell;
    for (int a = 0; a < 3; ++a) { d.h[a] = g.h[a]; d.S[a] = g.S[a]; }
    d.V = g.V;
    return d;
}

template <typename T> struct P3 { T *a[3]; };
template <typename T> struct C3 { const T *a[3]; };

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

__device__ __forceinline__ void coords(const GridD &g, int c, int &i, int &j, int &k) {
    i = c % g.nx;
    int r = c / g.nx;
    j = r % g.ny;
    k = r / g.ny;
}
__device__ __forceinline__ int flo(const GridD &g, int a, int i, int j, int k) {
    if (a == 0) return i + (g.nx + 1) * (j + g.ny * k);
    if (a == 1) return i + g.nx * (j + (g.ny + 1) * k);
    return i + g.nx * (j + g.ny * k);
}
__device__ __forceinline__ int fhi(const GridD &g, int a, int i, int j, int k) {
    if (a == 0) return flo(g, 0, i, j, k) + 1;
    if (a == 1) return flo(g, 1, i, j, k) + g.nx;
    return flo(g, 2, i, j, k) + g.nx * g.ny;
}
__device__ __forceinline__ int noff(const GridD &g, int a) { return a == 0 ? 1 : (a == 1 ? g.nx : g.nx * g.ny); }

// Decode face f of direction A into its fluid neighbours and type.
template <int A>
__device__ __forceinline__ int decode_face(const GridD &g, const uint32_t *__restrict__ info, int f, int &L, int &H) {
    int i, j, k, q, n;
    if (A == 0) { i = f % (g.nx + 1); int r = f / (g.nx + 1); j = r % g.ny; k = r / g.ny; q = i; n = g.nx; }
    else if (A == 1) { i = f % g.nx; int r = f / g.nx; j = r % (g.ny + 1); k = r / (g.ny + 1); q = j; n = g.ny; }
    else { i = f % g.nx; int r = f / g.nx; j = r % g.ny; k = r / g.ny; q = k; n = g.nz; }
    int off = A == 0 ? 1 : (A == 1 ? g.nx : g.nx * g.ny);
    int c = i + g.nx * (j + g.ny * k);
    L = -1; H = -1;
    if (q < n && (info[c] & INFO_FLUID)) {
        int t = ftype(info[c], A, 0);
        H = c;
        if (t == FT_INTERIOR) L = c - off;
        return t;
    }
    if (q > 0 && (info[c - off] & INFO_FLUID)) {
        L = c - off;
        return ftype(info[c - off], A, 1);
    }
    return FT_NONE;
}

// ---------------------------------------------------------------------------
// reductions (fixed grid, deterministic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (w == 0) {
        v = l < nw ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}
__device__ __forceinline__ double block_max(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (w == 0) {
        v = l < nw ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;
}

// out[slot] = sum (or max) of partials[0..nb)
static __global__ void k_final(const double *__restrict__ partials, int nb, double *__restrict__ out, int is_max) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v = is_max ? fmax(v, partials[b]) : v + partials[b];
    v = is_max ? block_max(v) : block_sum(v);
    if (threadIdx.x == 0) *out = v;
}

// ---------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_build_info(GridD g, const uint8_t *__restrict__ solid, uint32_t *__restrict__ info,
                             uint8_t *__restrict__ fluid) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    if (solid[c]) { info[c] = 0; fluid[c] = 0; return; }
    int ijk[3];
    coords(g, c, ijk[0], ijk[1], ijk[2]);
    int n[3] = {g.nx, g.ny, g.nz};
    uint32_t w = INFO_FLUID;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        for (int s = 0; s < 2; ++s) {
            int q = ijk[a] + (s ? 1 : -1);
            int t;
            if (q < 0) t = (a == 0) ? FT_INLET : FT_WALL;
            else if (q >= n[a]) t = (a == 0) ? FT_OUTLET : FT_WALL;
            else t = solid[c + (s ? 1 : -1) * noff(g, a)] ? FT_WALL : FT_INTERIOR;
            w |= (uint32_t)t << (3 * (2 * a + s));
        }
    }
    info[c] = w;
    fluid[c] = 1;
}

template <typename T>
__global__ void k_load_alpha(int n, const uint32_t *__restrict__ info, const double *__restrict__ src, T *__restrict__ dst) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    dst[c] = (info[c] & INFO_FLUID) ? (T)src[c] : T(0);
}

template <typename S, typename D>
__global__ void k_convert(int n, const S *__restrict__ src, D *__restrict__ dst) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) dst[c] = (D)src[c];
}

template <typename T>
__global__ void k_sum2(int n, const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = a[c] + b[c];
}

template <typename T>
__global__ void k_fill(int n, T *__restrict__ x, T v) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) x[c] = v;
}

// ---------------------------------------------------------------------------
// alpha transport: explicit Euler (Eq. alphaExp) with a vanLeer high-order
// flux, interface compression and a Zalesak flux-corrected-transport limiter
// ---------------------------------------------------------------------------
// Low-order (upwind) flux FL and antidiffusive flux AD of an interior face
// between fluid cells L (low) and H (high) of direction a.
template <typename T>
__device__ __forceinline__ void ho_flux(const uint32_t *__restrict__ info, const T *__restrict__ alpha, int a, int off,
                                        int L, int H, T ph, T nfv, T c_alpha, T &FL, T &AD) {
    int U, D, UU = -1;
    if (ph >= T(0)) {
        U = L; D = H;
        if (ftype(info[L], a, 0) == FT_INTERIOR) UU = L - off;
    } else {
        U = H; D = L;
        if (ftype(info[H], a, 1) == FT_INTERIOR) UU = H + off;
    }
    T aU = alpha[U], aD = alpha[D];
    T dc = aD - aU;
    T du = UU >= 0 ? (aU - alpha[UU]) : T(0);
    // vanLeer: aU + psi(r)/2 (aD - aU), psi = (r+|r|)/(1+|r|), r = du/dc
    T avl = (du * dc > T(0)) ? aU + du * dc / (du + dc) : aU;
    T flow = ph * aU;
    // compression flux phi_r alpha (1 - alpha), phi_r = c_alpha |phi| n_f
    T phir = c_alpha * tabs(ph) * nfv;
    T aLv = alpha[L], aHv = alpha[H];
    T fc = (phir >= T(0)) ? phir * aLv * (T(1) - aHv) : phir * aHv * (T(1) - aLv);
    T fhigh = ph * avl + fc;
    FL = flow;
    AD = fhigh - flow;
}

template <int DIM, typename T>
__global__ void k_transport_low(GridD g, const uint32_t *__restrict__ info, const T *__restrict__ alpha, C3<T> phi,
                                C3<T> nf, T c_alpha, T alpha_in, T rV, T *__restrict__ aL, T *__restrict__ Pp,
                                T *__restrict__ Pm) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) { aL[c] = T(0); Pp[c] = T(0); Pm[c] = T(0); return; }
    int i, j, k;
    coords(g, c, i, j, k);
    T out = T(0), pp = T(0), pm = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int t = ftype(inf, a, s);
            int f = s ? fhi(g, a, i, j, k) : flo(g, a, i, j, k);
            T ph = phi.a[a][f];
            T FL = T(0), AD = T(0);
            if (t == FT_INTERIOR) {
                int nb = s ? c + off : c - off;
                ho_flux<T>(info, alpha, a, off, s ? c : nb, s ? nb : c, ph, nf.a[a][f], c_alpha, FL, AD);
            } else if (t == FT_INLET) {
                FL = ph >= T(0) ? ph * alpha_in : ph * alpha[c];
            } else if (t == FT_OUTLET) {
                FL = ph * alpha[c];
            }
            out += s ? FL : -FL;
            T aout = s ? AD : -AD;
            if (aout > T(0)) pm += aout; else pp += -aout;
        }
    }
    aL[c] = alpha[c] - rV * out;
    Pp[c] = pp;
    Pm[c] = pm;
}

template <int DIM, typename T>
__global__ void k_transport_ratio(GridD g, const uint32_t *__restrict__ info, const T *__restrict__ alpha,
                                  const T *__restrict__ aL, const T *__restrict__ Pp, const T *__restrict__ Pm, T rV,
                                  T *__restrict__ Rp, T *__restrict__ Rm) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) { Rp[c] = T(0); Rm[c] = T(0); return; }
    T a0 = alpha[c], l0 = aL[c];
    T amax = a0 > l0 ? a0 : l0;
    T amin = a0 < l0 ? a0 : l0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (ftype(inf, a, s) != FT_INTERIOR) continue;
            int nb = s ? c + off : c - off;
            T an = alpha[nb], ln = aL[nb];
            if (an > amax) amax = an;
            if (ln > amax) amax = ln;
            if (an < amin) amin = an;
            if (ln < amin) amin = ln;
        }
    }
    if (amax > T(1)) amax = T(1);
    if (amin < T(0)) amin = T(0);
    T Qp = (amax - l0) / rV;
    T Qm = (l0 - amin) / rV;
    if (Qp < T(0)) Qp = T(0);
    if (Qm < T(0)) Qm = T(0);
    T pp = Pp[c], pm = Pm[c];
    Rp[c] = pp > T(0) ? (Qp / pp < T(1) ? Qp / pp : T(1)) : T(0);
    Rm[c] = pm > T(0) ? (Qm / pm < T(1) ? Qm / pm : T(1)) : T(0);
}

template <int DIM, typename T>
__global__ void k_transport_update(GridD g, const uint32_t *__restrict__ info, const T *__restrict__ alpha, C3<T> phi,
                                   C3<T> nf, T c_alpha, const T *__restrict__ aL, const T *__restrict__ Rp,
                                   const T *__restrict__ Rm, T rV, T *__restrict__ alpha_new) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) { alpha_new[c] = T(0); return; }
    int i, j, k;
    coords(g, c, i, j, k);
    T out = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (ftype(inf, a, s) != FT_INTERIOR) continue;
            int f = s ? fhi(g, a, i, j, k) : flo(g, a, i, j, k);
            int nb = s ? c + off : c - off;
            int L = s ? c : nb, H = s ? nb : c;
            T FL, AD;
            ho_flux<T>(info, alpha, a, off, L, H, phi.a[a][f], nf.a[a][f], c_alpha, FL, AD);
            T lam;
            if (AD >= T(0)) lam = Rm[L] < Rp[H] ? Rm[L] : Rp[H];
            else lam = Rm[H] < Rp[L] ? Rm[H] : Rp[L];
            T fl = lam * AD;
            out += s ? fl : -fl;
        }
    }
    alpha_new[c] = aL[c] - rV * out;
}

// ---------------------------------------------------------------------------
// interface: smoothed alpha, face normals with the contact angle, curvature
// (Section 2.1; wall condition of Eqs. VOFd / VOFc)
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void k_smooth(GridD g, const uint32_t *__restrict__ info, const T *__restrict__ src, T *__restrict__ dst) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) { dst[c] = T(0); return; }
    T num = T(0), den = T(0);
    T x = src[c];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
        T Sa = (T)g.S[a];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            T af = ftype(inf, a, s) == FT_INTERIOR ? T(0.5) * (x + src[s ? c + off : c - off]) : x;
            num += af * Sa;
            den += Sa;
        }
    }
    dst[c] = num / den;
}

template <int DIM, typename T>
__device__ __forceinline__ T gauss_grad(const GridD &g, const uint32_t *__restrict__ info, const T *__restrict__ x, int c,
                                        int b) {
    uint32_t inf = info[c];
    int off = noff(g, b);
    T xc = x[c];
    T f0 = ftype(inf, b, 0) == FT_INTERIOR ? T(0.5) * (xc + x[c - off]) : xc;
    T f1 = ftype(inf, b, 1) == FT_INTERIOR ? T(0.5) * (xc + x[c + off]) : xc;
    return (f1 - f0) / (T)g.h[b];
}

template <int DIM, int A, typename T>
__global__ void k_normals(GridD g, int nfaces, const uint32_t *__restrict__ info, const T *__restrict__ as, T ct, T deltaN,
                          T *__restrict__ nfA) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfaces) return;
    int L, H;
    int t = decode_face<A>(g, info, f, L, H);
    T n = T(0);
    if (t == FT_INTERIOR) {
        T gv[3] = {T(0), T(0), T(0)};
        gv[A] = (as[H] - as[L]) / (T)g.h[A];
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            if (b == A) continue;
            gv[b] = T(0.5) * (gauss_grad<DIM, T>(g, info, as, L, b) + gauss_grad<DIM, T>(g, info, as, H, b));
        }
        T mag = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b) mag += gv[b] * gv[b];
        mag = sqrt(mag);
        n = gv[A] / (mag + deltaN);
    } else if (t == FT_WALL) {
        n = (L >= 0) ? ct : -ct;   // n . n_wall = cos(theta), n_wall out of the fluid cell
    }
    nfA[f] = n;
}

template <int DIM, typename T>
__global__ void k_curvature(GridD g, const uint32_t *__restrict__ info, C3<T> nf, T *__restrict__ kappa) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    if (!(info[c] & INFO_FLUID)) { kappa[c] = T(0); return; }
    int i, j, k;
    coords(g, c, i, j, k);
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) acc += (nf.a[a][fhi(g, a, i, j, k)] - nf.a[a][flo(g, a, i, j, k)]) / (T)g.h[a];
    kappa[c] = -acc;
}

// ---------------------------------------------------------------------------
// PISO (Section 2.2 with Eqs. NSE1d / NSEc, advective form of ddt + convection)
// ---------------------------------------------------------------------------
template <typename T> struct Fluid { T rho1, rho2, mu1, mu2; };
template <typename T> __device__ __forceinline__ T mix(T al, T p1, T p2) { return al * p1 + (T(1) - al) * p2; }

template <int DIM, typename T>
__global__ void k_rA(GridD g, const uint32_t *__restrict__ info, const T *__restrict__ alpha, C3<T> phic, Fluid<T> fl,
                     T dt, T *__restrict__ rA) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) { rA[c] = T(0); return; }
    int i, j, k;
    coords(g, c, i, j, k);
    T al = alpha[c];
    T rho = mix(al, fl.rho1, fl.rho2), mu = mix(al, fl.mu1, fl.mu2);
    T acc = T(0), cin = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
        T Sa = (T)g.S[a], ha = (T)g.h[a];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int t = ftype(inf, a, s);
            if (t == FT_INTERIOR) {
                T mun = mix(alpha[s ? c + off : c - off], fl.mu1, fl.mu2);
                acc += T(0.5) * (mu + mun) * Sa / ha;
            } else if (t == FT_WALL || t == FT_INLET) {
                acc += mu * Sa / (T(0.5) * ha);
            }
            if (t == FT_INTERIOR || t == FT_INLET) {
                T fo = (s ? T(1) : T(-1)) * phic.a[a][s ? fhi(g, a, i, j, k) : flo(g, a, i, j, k)];
                if (fo < T(0)) cin += -fo;   // inflow: implicit upwind part of convection
            }
        }
    }
    rA[c] = T(1) / (rho / dt + (acc + rho * cin) / (T)g.V);
}

// pressure-operator coefficients c_f (MG level 0) and CSF face forces
template <int A, typename T>
__global__ void k_face_coeffs(GridD g, int nfaces, const uint32_t *__restrict__ info, const T *__restrict__ rA,
                              const T *__restrict__ kappa, const T *__restrict__ alpha, T sigma, int has_st,
                              T *__restrict__ cf, T *__restrict__ fst) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfaces) return;
    int L, H;
    int t = decode_face<A>(g, info, f, L, H);
    T Sa = (T)g.S[A], ha = (T)g.h[A];
    T c = T(0), fs = T(0);
    if (t == FT_INTERIOR) {
        c = T(0.5) * (rA[L] + rA[H]) * Sa / ha;
        if (has_st) fs = sigma * T(0.5) * (kappa[L] + kappa[H]) * (alpha[H] - alpha[L]) / ha;
    } else if (t == FT_OUTLET) {
        c = rA[L] * Sa / (T(0.5) * ha);
    }
    cf[f] = c;
    fst[f] = fs;
}

// Gauss gradients of the velocity iterate: G[comp*3 + dir]
template <int DIM, typename T>
__global__ void k_vel_grad(GridD g, const uint32_t *__restrict__ info, C3<T> v, T vin0, P3<T> G0, P3<T> G1, P3<T> G2) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) return;
    T *Gr[3][3] = {{G0.a[0], G0.a[1], G0.a[2]}, {G1.a[0], G1.a[1], G1.a[2]}, {G2.a[0], G2.a[1], G2.a[2]}};
#pragma unroll
    for (int comp = 0; comp < DIM; ++comp) {
        T vc = v.a[comp][c];
        T vin = comp == 0 ? vin0 : T(0);
#pragma unroll
        for (int dir = 0; dir < DIM; ++dir) {
            int off = noff(g, dir);
            T fv[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                int t = ftype(inf, dir, s);
                if (t == FT_INTERIOR) fv[s] = T(0.5) * (vc + v.a[comp][s ? c + off : c - off]);
                else if (t == FT_INLET) fv[s] = vin;
                else if (t == FT_OUTLET) fv[s] = vc;
                else fv[s] = T(0);
            }
            Gr[comp][dir][c] = (fv[1] - fv[0]) / (T)g.h[dir];
        }
    }
}

// HbyA = H/A: old-time term, explicit neighbour part of the viscous Laplacian,
// linear-upwind convection (advective form) and the transpose viscous term.
template <int DIM, typename T>
__global__ void k_momentum_H(GridD g, const uint32_t *__restrict__ info, C3<T> v, C3<T> vold, C3<T> phic,
                             const T *__restrict__ alpha, const T *__restrict__ rA, Fluid<T> fl, T vin0, T dt,
                             C3<T> G0, C3<T> G1, C3<T> G2, P3<T> hbya) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) {
#pragma unroll
        for (int comp = 0; comp < DIM; ++comp) hbya.a[comp][c] = T(0);
        return;
    }
    const T *Gr[3][3] = {{G0.a[0], G0.a[1], G0.a[2]}, {G1.a[0], G1.a[1], G1.a[2]}, {G2.a[0], G2.a[1], G2.a[2]}};
    int i, j, k;
    coords(g, c, i, j, k);
    T al = alpha[c];
    T rho = mix(al, fl.rho1, fl.rho2), mu = mix(al, fl.mu1, fl.mu2);
    T rAc = rA[c];
#pragma unroll
    for (int comp = 0; comp < DIM; ++comp) {
        T vc = v.a[comp][c];
        T vin = comp == 0 ? vin0 : T(0);
        T Hc = rho * vold.a[comp][c] / dt;
        T lap = T(0), conv = T(0), tr = T(0), inflow = T(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            int off = noff(g, a);
            T Sa = (T)g.S[a], ha = (T)g.h[a];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                int t = ftype(inf, a, s);
                T sg = s ? T(1) : T(-1);
                int f = s ? fhi(g, a, i, j, k) : flo(g, a, i, j, k);
                if (t == FT_INTERIOR) {
                    int nb = s ? c + off : c - off;
                    T mun = mix(alpha[nb], fl.mu1, fl.mu2);
                    T muf = T(0.5) * (mu + mun);
                    lap += muf * Sa / ha * v.a[comp][nb];
                    int L = s ? c : nb, Hh = s ? nb : c;
                    T pc = phic.a[a][f];
                    T vf, vu;
                    if (pc >= T(0)) { vu = v.a[comp][L]; vf = vu + T(0.5) * ha * Gr[comp][a][L]; }
                    else { vu = v.a[comp][Hh]; vf = vu - T(0.5) * ha * Gr[comp][a][Hh]; }
                    T fo = sg * pc;
                    if (fo < T(0)) inflow += -fo * v.a[comp][nb];
                    conv += fo * (vf - vu);
                    T dvdx = T(0.5) * (Gr[a][comp][c] + Gr[a][comp][nb]);
                    tr += sg * muf * Sa * dvdx;
                } else if (t == FT_WALL) {
                    tr += sg * mu * Sa * Gr[a][comp][c];
                } else if (t == FT_INLET) {
                    lap += mu * Sa / (T(0.5) * ha) * vin;
                    T fo = sg * phic.a[a][f];
                    if (fo < T(0)) inflow += -fo * vin;
                    else conv += fo * (vin - vc);
                    tr += sg * mu * Sa * Gr[a][comp][c];
                } else if (t == FT_OUTLET) {
                    tr += sg * mu * Sa * Gr[a][comp][c];
                }
            }
        }
        Hc += (lap + rho * (inflow - conv) + tr) / (T)g.V;
        hbya.a[comp][c] = rAc * Hc;
    }
}

template <int A, typename T>
__global__ void k_phistar(GridD g, int nfaces, const uint32_t *__restrict__ info, const T *__restrict__ hbyaA,
                          const T *__restrict__ rA, const T *__restrict__ fst, T vinA, T *__restrict__ phis) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfaces) return;
    int L, H;
    int t = decode_face<A>(g, info, f, L, H);
    T Sa = (T)g.S[A];
    T ps = T(0);
    if (t == FT_INTERIOR) ps = T(0.5) * (hbyaA[L] + hbyaA[H]) * Sa + T(0.5) * (rA[L] + rA[H]) * fst[f] * Sa;
    else if (t == FT_INLET) ps = vinA * Sa;
    else if (t == FT_OUTLET) ps = hbyaA[L] * Sa;
    phis[f] = ps;
}

// b = -div(phi*) (double)
template <int DIM, typename T>
__global__ void k_rhs(GridD g, const uint32_t *__restrict__ info, C3<T> phis, double *__restrict__ b) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    if (!(info[c] & INFO_FLUID)) { b[c] = 0.0; return; }
    int i, j, k;
    coords(g, c, i, j, k);
    double div = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        div += -(double)phis.a[a][flo(g, a, i, j, k)];
        div += (double)phis.a[a][fhi(g, a, i, j, k)];
    }
    b[c] = -div;
}

// (M q)_P = sum_f c_f (q_P - q_N) + sum_outlet c_f q_P
template <int DIM, typename T>
__device__ __forceinline__ double poisson_row(const GridD &g, uint32_t inf, int c, int i, int j, int k, C3<T> cf,
                                              const double *__restrict__ q) {
    double acc = 0.0;
    double qc = q[c];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int t = ftype(inf, a, s);
            if (t == FT_INTERIOR) {
                int f = s ? fhi(g, a, i, j, k) : flo(g, a, i, j, k);
                acc += (double)cf.a[a][f] * (qc - q[s ? c + off : c - off]);
            } else if (t == FT_OUTLET) {
                acc += (double)cf.a[a][fhi(g, a, i, j, k)] * qc;
            }
        }
    }
    return acc;
}

template <int DIM, typename T>
__device__ __forceinline__ double outlet_sum(const GridD &g, uint32_t inf, int i, int j, int k, C3<T> cf) {
    return ftype(inf, 0, 1) == FT_OUTLET ? (double)cf.a[0][fhi(g, 0, i, j, k)] : 0.0;
}

// partial sums for the normalised residual: res = |b - Mq|, nrm = |Mq - M qbar| + |b - M qbar|
template <int DIM, typename T>
__global__ void k_normres(GridD g, const uint32_t *__restrict__ info, C3<T> cf, const double *__restrict__ q,
                          const double *__restrict__ b, const double *__restrict__ scal, double inv_nf,
                          double *__restrict__ part_res, double *__restrict__ part_nrm) {
    double qbar = scal[S_QSUM] * inv_nf;
    double res = 0.0, nrm = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
        uint32_t inf = info[c];
        if (!(inf & INFO_FLUID)) continue;
        int i, j, k;
        coords(g, c, i, j, k);
        double Mq = poisson_row<DIM, T>(g, inf, c, i, j, k, cf, q);
        double Mqbar = qbar * outlet_sum<DIM, T>(g, inf, i, j, k, cf);
        res += fabs(b[c] - Mq);
        nrm += fabs(Mq - Mqbar) + fabs(b[c] - Mqbar);
    }
    res = block_sum(res);
    nrm = block_sum(nrm);
    if (threadIdx.x == 0) { part_res[blockIdx.x] = res; part_nrm[blockIdx.x] = nrm; }
}

template <typename T>
__global__ void k_sum_field(int n, const T *__restrict__ x, double scale, double *__restrict__ part) {
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) acc += (double)x[c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc * scale;
}

// flux correction phi = phi* - c_f (q_H - q_L)
template <int A, typename T>
__global__ void k_flux_correct(GridD g, int nfaces, const uint32_t *__restrict__ info, const T *__restrict__ phis,
                               const T *__restrict__ cf, const double *__restrict__ q, T *__restrict__ phi) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfaces) return;
    int L, H;
    int t = decode_face<A>(g, info, f, L, H);
    double ps = (double)phis[f];
    double out = ps;
    if (t == FT_INTERIOR) out = ps - (double)cf[f] * (q[H] - q[L]);
    else if (t == FT_OUTLET) out = ps - (double)cf[f] * (0.0 - q[L]);
    phi[f] = (T)out;
}

// v = HbyA + rA * reconstruct(face accelerations)
template <int DIM, typename T>
__global__ void k_vel_correct(GridD g, const uint32_t *__restrict__ info, C3<T> hbya, const T *__restrict__ rA,
                              C3<T> fst, const double *__restrict__ q, P3<T> v) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    uint32_t inf = info[c];
    if (!(inf & INFO_FLUID)) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) v.a[a][c] = T(0);
        return;
    }
    int i, j, k;
    coords(g, c, i, j, k);
    double qc = q[c];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
        double ha = g.h[a];
        double gs = 0.0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int t = ftype(inf, a, s);
            if (t == FT_INTERIOR) {
                int nb = s ? c + off : c - off;
                int f = s ? fhi(g, a, i, j, k) : flo(g, a, i, j, k);
                double qL = s ? qc : q[nb], qH = s ? q[nb] : qc;
                gs += (double)fst.a[a][f] - (qH - qL) / ha;
            } else if (t == FT_OUTLET) {
                gs += -(0.0 - qc) / (0.5 * ha);
            }
        }
        v.a[a][c] = (T)((double)hbya.a[a][c] + (double)rA[c] * 0.5 * gs);
    }
}

// u_sum += v; partial max |v - vold|
template <int DIM, typename T>
__global__ void k_relax_accum(int n, const uint32_t *__restrict__ info, C3<T> v, C3<T> vold, P3<double> usum,
                              double *__restrict__ part) {
    double m = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        if (!(info[c] & INFO_FLUID)) continue;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double x = (double)v.a[a][c];
            usum.a[a][c] += x;
            m = fmax(m, fabs(x - (double)vold.a[a][c]));
        }
    }
    m = block_max(m);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

// ---------------------------------------------------------------------------
// CG (FP64 vectors)
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void k_cg_init(GridD g, const uint32_t *__restrict__ info, C3<T> cf, const double *__restrict__ q,
                          const double *__restrict__ b, double *__restrict__ r, double *__restrict__ part_bb,
                          double *__restrict__ part_rr) {
    double bb = 0.0, rr = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
        uint32_t inf = info[c];
        if (!(inf & INFO_FLUID)) { r[c] = 0.0; continue; }
        int i, j, k;
        coords(g, c, i, j, k);
        double rc = b[c] - poisson_row<DIM, T>(g, inf, c, i, j, k, cf, q);
        r[c] = rc;
        bb += b[c] * b[c];
        rr += rc * rc;
    }
    bb = block_sum(bb);
    rr = block_sum(rr);
    if (threadIdx.x == 0) { part_bb[blockIdx.x] = bb; part_rr[blockIdx.x] = rr; }
}

template <int DIM, typename T>
__global__ void k_cg_apply_dot(GridD g, const uint32_t *__restrict__ info, C3<T> cf, const double *__restrict__ p,
                               double *__restrict__ Ap, double *__restrict__ part) {
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
        uint32_t inf = info[c];
        if (!(inf & INFO_FLUID)) { Ap[c] = 0.0; continue; }
        int i, j, k;
        coords(g, c, i, j, k);
        double y = poisson_row<DIM, T>(g, inf, c, i, j, k, cf, p);
        Ap[c] = y;
        acc += p[c] * y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

static __global__ void k_cg_update(int n, const double *__restrict__ scal, int slot_rz, double *__restrict__ q,
                            double *__restrict__ r, const double *__restrict__ p, const double *__restrict__ Ap,
                            double *__restrict__ part) {
    double al = scal[slot_rz] / scal[S_PAP];
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        q[c] += al * p[c];
        double rc = r[c] - al * Ap[c];
        r[c] = rc;
        acc += rc * rc;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

static __global__ void k_dot(int n, const double *__restrict__ x, const double *__restrict__ y, double *__restrict__ part) {
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) acc += x[c] * y[c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// p = z + beta p, beta = scal[new]/scal[old] (beta = 0 when first)
static __global__ void k_cg_pupdate(int n, const double *__restrict__ scal, int slot_new, int slot_old, int first,
                             const double *__restrict__ z, double *__restrict__ p) {
    double be = first ? 0.0 : scal[slot_new] / scal[slot_old];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        p[c] = first ? z[c] : z[c] + be * p[c];
}

// ---------------------------------------------------------------------------
// geometric multigrid (preconditioner): piecewise-constant transfers, coarse
// operators from summed fine face coefficients (x 1/2 across a coarsened
// direction), red-black Gauss-Seidel smoothing
// ---------------------------------------------------------------------------
template <typename M> struct MG3 { const M *a[3]; };

template <int DIM, typename M>
__device__ __forceinline__ M mg_offdiag(const GridD &g, MG3<M> c, const M *__restrict__ x, int cell, int i, int j,
                                        int k) {
    M acc = M(0);
    int ijk[3] = {i, j, k};
    int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int off = noff(g, a);
        if (ijk[a] > 0) acc += c.a[a][flo(g, a, i, j, k)] * x[cell - off];
        if (ijk[a] < n[a] - 1) acc += c.a[a][fhi(g, a, i, j, k)] * x[cell + off];
    }
    return acc;
}

template <int DIM, typename M>
__global__ void k_mg_rbgs(GridD g, const uint8_t *__restrict__ fluid, MG3<M> c, const M *__restrict__ diag,
                          M *__restrict__ x, const M *__restrict__ b, int colour) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.ncell) return;
    int i, j, k;
    coords(g, cell, i, j, k);
    if (((i + j + k) & 1) != colour) return;
    M d = diag[cell];
    if (!fluid[cell] || d <= M(0)) return;
    x[cell] = (b[cell] + mg_offdiag<DIM, M>(g, c, x, cell, i, j, k)) / d;
}

template <int DIM, typename M>
__global__ void k_mg_residual(GridD g, const uint8_t *__restrict__ fluid, MG3<M> c, const M *__restrict__ diag,
                              const M *__restrict__ x, const M *__restrict__ b, M *__restrict__ res) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.ncell) return;
    if (!fluid[cell]) { res[cell] = M(0); return; }
    int i, j, k;
    coords(g, cell, i, j, k);
    res[cell] = b[cell] - (diag[cell] * x[cell] - mg_offdiag<DIM, M>(g, c, x, cell, i, j, k));
}

// coarse b = sum of children residuals; coarse x = 0
template <typename M>
__global__ void k_mg_restrict(GridD gf, GridD gc, int rx, int ry, int rz, const M *__restrict__ res,
                              M *__restrict__ bc, M *__restrict__ xc) {
    int C = blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= gc.ncell) return;
    int I, J, K;
    coords(gc, C, I, J, K);
    M acc = M(0);
    for (int oz = 0; oz < rz; ++oz) {
        int k = K * rz + oz;
        if (k >= gf.nz) break;
        for (int oy = 0; oy < ry; ++oy) {
            int j = J * ry + oy;
            if (j >= gf.ny) break;
            for (int ox = 0; ox < rx; ++ox) {
                int i = I * rx + ox;
                if (i >= gf.nx) break;
                acc += res[i + gf.nx * (j + gf.ny * k)];
            }
        }
    }
    bc[C] = acc;
    xc[C] = M(0);
}

template <typename M>
__global__ void k_mg_prolong(GridD gf, GridD gc, int rx, int ry, int rz, const uint8_t *__restrict__ fluid,
                             const M *__restrict__ xc, M *__restrict__ x) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= gf.ncell) return;
    if (!fluid[cell]) return;
    int i, j, k;
    coords(gf, cell, i, j, k);
    x[cell] += xc[(i / rx) + gc.nx * ((j / ry) + gc.ny * (k / rz))];
}

static __global__ void k_mg_fluid_coarsen(GridD gf, GridD gc, int rx, int ry, int rz, const uint8_t *__restrict__ ff,
                                   uint8_t *__restrict__ fc) {
    int C = blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= gc.ncell) return;
    int I, J, K;
    coords(gc, C, I, J, K);
    uint8_t any = 0;
    for (int oz = 0; oz < rz; ++oz)
        for (int oy = 0; oy < ry; ++oy)
            for (int ox = 0; ox < rx; ++ox) {
                int i = I * rx + ox, j = J * ry + oy, k = K * rz + oz;
                if (i < gf.nx && j < gf.ny && k < gf.nz && ff[i + gf.nx * (j + gf.ny * k)]) any = 1;
            }
    fc[C] = any;
}

// coarse face coefficient of direction A
template <int A, typename M>
__global__ void k_mg_coarse_coeff(GridD gf, GridD gc, int nfaces, int rx, int ry, int rz, const M *__restrict__ cfine,
                                  M *__restrict__ ccoarse) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfaces) return;
    int I, J, K;
    if (A == 0) { I = f % (gc.nx + 1); int r = f / (gc.nx + 1); J = r % gc.ny; K = r / gc.ny; }
    else if (A == 1) { I = f % gc.nx; int r = f / gc.nx; J = r % (gc.ny + 1); K = r / (gc.ny + 1); }
    else { I = f % gc.nx; int r = f / gc.nx; J = r % gc.ny; K = r / gc.ny; }
    int rr[3] = {rx, ry, rz};
    int nfn[3] = {gf.nx, gf.ny, gf.nz};
    int base[3] = {I, J, K};
    // fine face coordinate along A, children ranges across
    int lo[3], cnt[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (b == A) {
            lo[b] = rr[b] == 2 ? min(2 * base[b], nfn[b]) : base[b];
            cnt[b] = 1;
        } else {
            lo[b] = base[b] * rr[b];
            cnt[b] = min(rr[b], nfn[b] - lo[b]);
        }
    }
    M acc = M(0);
    for (int oz = 0; oz < cnt[2]; ++oz)
        for (int oy = 0; oy < cnt[1]; ++oy)
            for (int ox = 0; ox < cnt[0]; ++ox)
                acc += cfine[flo(gf, A, lo[0] + ox, lo[1] + oy, lo[2] + oz)];
    ccoarse[f] = rr[A] == 2 ? M(0.5) * acc : acc;
}

template <int DIM, typename M>
__global__ void k_mg_diag(GridD g, const uint8_t *__restrict__ fluid, MG3<M> c, M *__restrict__ diag) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.ncell) return;
    if (!fluid[cell]) { diag[cell] = M(0); return; }
    int i, j, k;
    coords(g, cell, i, j, k);
    M acc = M(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) acc += c.a[a][flo(g, a, i, j, k)] + c.a[a][fhi(g, a, i, j, k)];
    diag[cell] = acc;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
#define OSCAR_LAUNCH_CHECK()                                        \
    do {                                                            \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) {                                    \
            fprintf(stderr, "oscar: CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return OSCAR_E_CUDA;                                    \
        }                                                           \
    } while (0)

inline int nblk(long long n) { return (int)((n + BS - 1) / BS); }

template <typename T> struct Impl {
    using M = T;
    static T *tp(void *p) { return (T *)p; }

    static int final_sum(Instance &I, int slot_part, int slot_out, bool is_max = false) {
        k_final<<<1, 1024, 0, I.stream>>>(I.partials + slot_part * kRedBlocks, kRedBlocks, I.scal + slot_out,
                                          is_max ? 1 : 0), ++I.nlaunch;
        return 0;
    }
    static int read_scalars(Instance &I) {
        if (cudaMemcpyAsync(I.scal_host, I.scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, I.stream) !=
            cudaSuccess)
            return OSCAR_E_CUDA;
        return sync_bounded(I.stream, kSyncTimeoutSec);
    }
    static C3<T> c3(void *const *p) { C3<T> r; for (int a = 0; a < 3; ++a) r.a[a] = (const T *)p[a]; return r; }
    static P3<T> p3(void *const *p) { P3<T> r; for (int a = 0; a < 3; ++a) r.a[a] = (T *)p[a]; return r; }

    // --- transport ---------------------------------------------------------
    template <int DIM>
    static int transport_d(Instance &I, void *const *phi, double dt) {
        GridD g = to_dev(I.g);
        T rV = (T)(dt / I.g.V);
        int nb = nblk(g.ncell);
        int ps = prof_begin(I, OSCAR_KID_TRANSPORT);
        k_transport_low<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, tp(I.alpha), c3(phi), c3(I.nf), (T)I.P.c_alpha,
                                                         (T)I.P.alpha_inlet, rV, tp(I.aL), tp(I.Pp), tp(I.Pm)), ++I.nlaunch;
        k_transport_ratio<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, tp(I.alpha), tp(I.aL), tp(I.Pp), tp(I.Pm), rV,
                                                           tp(I.Rp), tp(I.Rm)), ++I.nlaunch;
        k_transport_update<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, tp(I.alpha), c3(phi), c3(I.nf),
                                                            (T)I.P.c_alpha, tp(I.aL), tp(I.Rp), tp(I.Rm), rV,
                                                            tp(I.alpha_new)), ++I.nlaunch;
        prof_end(I, ps);
        OSCAR_LAUNCH_CHECK();
        return 0;
    }
    static int transport(Instance &I, void *const *phi, double dt) {
        return I.g.dim == 3 ? transport_d<3>(I, phi, dt) : transport_d<2>(I, phi, dt);
    }

    // --- interface ---------------------------------------------------------
    template <int DIM>
    static int interface_d(Instance &I, void *alpha) {
        GridD g = to_dev(I.g);
        int nb = nblk(g.ncell);
        void *src = alpha;
        for (int pass = 0; pass < I.P.n_smooth; ++pass) {
            void *dst = (pass % 2 == 0) ? I.alpha_s : I.alpha_tmp;
            k_smooth<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, tp(src), tp(dst)), ++I.nlaunch;
            src = dst;
        }
        const T *as = tp(src);
        T ct = (T)I.cos_theta, dn = (T)I.deltaN;
        k_normals<DIM, 0, T><<<nblk(I.g.nf[0]), BS, 0, I.stream>>>(g, I.g.nf[0], I.info, as, ct, dn, tp(I.nf[0])), ++I.nlaunch;
        k_normals<DIM, 1, T><<<nblk(I.g.nf[1]), BS, 0, I.stream>>>(g, I.g.nf[1], I.info, as, ct, dn, tp(I.nf[1])), ++I.nlaunch;
        if (DIM == 3)
            k_normals<DIM, 2, T><<<nblk(I.g.nf[2]), BS, 0, I.stream>>>(g, I.g.nf[2], I.info, as, ct, dn, tp(I.nf[2])), ++I.nlaunch;
        k_curvature<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, c3(I.nf), tp(I.kappa)), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return 0;
    }
    static int interface_(Instance &I, void *alpha) {
        return I.g.dim == 3 ? interface_d<3>(I, alpha) : interface_d<2>(I, alpha);
    }

    // --- multigrid -----------------------------------------------------------
    template <int DIM>
    static int mg_coeffs_d(Instance &I) {
        for (int l = 0; l < I.nlev; ++l) {
            Level &L = I.lev[l];
            GridD g = to_dev(L.g);
            if (l > 0) {
                Level &F = I.lev[l - 1];
                GridD gf = to_dev(F.g);
                k_mg_coarse_coeff<0, M><<<nblk(L.g.nf[0]), BS, 0, I.stream>>>(gf, g, L.g.nf[0], F.r[0], F.r[1], F.r[2],
                                                                          (const M *)F.c[0], (M *)L.c[0]), ++I.nlaunch;
                k_mg_coarse_coeff<1, M><<<nblk(L.g.nf[1]), BS, 0, I.stream>>>(gf, g, L.g.nf[1], F.r[0], F.r[1], F.r[2],
                                                                          (const M *)F.c[1], (M *)L.c[1]), ++I.nlaunch;
                if (DIM == 3)
                    k_mg_coarse_coeff<2, M><<<nblk(L.g.nf[2]), BS, 0, I.stream>>>(gf, g, L.g.nf[2], F.r[0], F.r[1],
                                                                              F.r[2], (const M *)F.c[2], (M *)L.c[2]), ++I.nlaunch;
            }
            MG3<M> c;
            for (int a = 0; a < 3; ++a) c.a[a] = (const M *)L.c[a];
            k_mg_diag<DIM, M><<<nblk(g.ncell), BS, 0, I.stream>>>(g, L.fluid, c, (M *)L.diag), ++I.nlaunch;
        }
        OSCAR_LAUNCH_CHECK();
        return 0;
    }

    template <int DIM>
    static void smooth_level(Instance &I, int l, int colour) {
        Level &L = I.lev[l];
        GridD g = to_dev(L.g);
        MG3<M> c;
        for (int a = 0; a < 3; ++a) c.a[a] = (const M *)L.c[a];
        int ps = l == 0 ? prof_begin(I, OSCAR_KID_RBGS0) : -1;
        k_mg_rbgs<DIM, M><<<nblk(g.ncell), BS, 0, I.stream>>>(g, L.fluid, c, (const M *)L.diag, (M *)L.x,
                                                              (const M *)L.b, colour), ++I.nlaunch;
        prof_end(I, ps);
    }

    // z = V-cycle(r)
    template <int DIM>
    static int vcycle_d(Instance &I, const double *r, double *z) {
        int n0 = I.g.ncell;
        k_convert<double, M><<<nblk(n0), BS, 0, I.stream>>>(n0, r, (M *)I.lev[0].b), ++I.nlaunch;
        k_fill<M><<<nblk(n0), BS, 0, I.stream>>>(n0, (M *)I.lev[0].x, M(0)), ++I.nlaunch;
        int nu = I.mg_nu;
        for (int l = 0; l < I.nlev - 1; ++l) {
            Level &L = I.lev[l], &C = I.lev[l + 1];
            for (int s = 0; s < nu; ++s) { smooth_level<DIM>(I, l, 0); smooth_level<DIM>(I, l, 1); }
            GridD g = to_dev(L.g), gc = to_dev(C.g);
            MG3<M> c;
            for (int a = 0; a < 3; ++a) c.a[a] = (const M *)L.c[a];
            int ps = l == 0 ? prof_begin(I, OSCAR_KID_RESID0) : -1;
            k_mg_residual<DIM, M><<<nblk(g.ncell), BS, 0, I.stream>>>(g, L.fluid, c, (const M *)L.diag,
                                                                      (const M *)L.x, (const M *)L.b, (M *)L.res), ++I.nlaunch;
            prof_end(I, ps);
            k_mg_restrict<M><<<nblk(gc.ncell), BS, 0, I.stream>>>(g, gc, L.r[0], L.r[1], L.r[2], (const M *)L.res,
                                                                  (M *)C.b, (M *)C.x), ++I.nlaunch;
        }
        int lc = I.nlev - 1;
        for (int s = 0; s < I.mg_coarse_sweeps; ++s) { smooth_level<DIM>(I, lc, 0); smooth_level<DIM>(I, lc, 1); }
        for (int s = 0; s < I.mg_coarse_sweeps; ++s) { smooth_level<DIM>(I, lc, 1); smooth_level<DIM>(I, lc, 0); }
        for (int l = I.nlev - 2; l >= 0; --l) {
            Level &L = I.lev[l], &C = I.lev[l + 1];
            GridD g = to_dev(L.g), gc = to_dev(C.g);
            k_mg_prolong<M><<<nblk(g.ncell), BS, 0, I.stream>>>(g, gc, L.r[0], L.r[1], L.r[2], L.fluid,
                                                                (const M *)C.x, (M *)L.x), ++I.nlaunch;
            for (int s = 0; s < nu; ++s) { smooth_level<DIM>(I, l, 1); smooth_level<DIM>(I, l, 0); }
        }
        k_convert<M, double><<<nblk(n0), BS, 0, I.stream>>>(n0, (const M *)I.lev[0].x, z), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return 0;
    }

    // PCG for M q = b; returns iterations (>=0) or a negative error code.
    template <int DIM>
    static int pcg_d(Instance &I, double *q, const double *b, int *not_conv) {
        GridD g = to_dev(I.g);
        C3<T> cf = c3(I.lev[0].c);
        int n = g.ncell;
        double *part = I.partials;
        k_cg_init<DIM, T><<<kRedBlocks, BS, 0, I.stream>>>(g, I.info, cf, q, b, I.cg_r, part, part + kRedBlocks), ++I.nlaunch;
        final_sum(I, 0, S_BB);
        final_sum(I, 1, S_RR);
        OSCAR_LAUNCH_CHECK();
        int rc = read_scalars(I);
        if (rc) return rc;
        double bn = sqrt(I.scal_host[S_BB]), rn = sqrt(I.scal_host[S_RR]);
        if (!isfinite(bn) || !isfinite(rn)) return OSCAR_E_NAN;
        double target = I.P.cg_rtol * (bn > 0.0 ? bn : rn);
        if (rn <= target) return 0;
        vcycle_d<DIM>(I, I.cg_r, I.cg_z);
        k_dot<<<kRedBlocks, BS, 0, I.stream>>>(n, I.cg_r, I.cg_z, part), ++I.nlaunch;
        int cur = S_RZ0, nxt = S_RZ1;
        final_sum(I, 0, cur);
        k_cg_pupdate<<<kRedBlocks, BS, 0, I.stream>>>(n, I.scal, cur, cur, 1, I.cg_z, I.cg_p), ++I.nlaunch;
        int it;
        for (it = 1; it <= I.P.cg_maxit; ++it) {
            int ps = prof_begin(I, OSCAR_KID_CG_APPLY);
            k_cg_apply_dot<DIM, T><<<kRedBlocks, BS, 0, I.stream>>>(g, I.info, cf, I.cg_p, I.cg_Ap, part), ++I.nlaunch;
            prof_end(I, ps);
            final_sum(I, 0, S_PAP);
            k_cg_update<<<kRedBlocks, BS, 0, I.stream>>>(n, I.scal, cur, q, I.cg_r, I.cg_p, I.cg_Ap, part), ++I.nlaunch;
            final_sum(I, 0, S_RR);
            OSCAR_LAUNCH_CHECK();
            rc = read_scalars(I);
            if (rc) return rc;
            rn = sqrt(I.scal_host[S_RR]);
            if (!isfinite(rn)) return OSCAR_E_NAN;
            if (rn <= target) break;
            vcycle_d<DIM>(I, I.cg_r, I.cg_z);
            k_dot<<<kRedBlocks, BS, 0, I.stream>>>(n, I.cg_r, I.cg_z, part), ++I.nlaunch;
            final_sum(I, 0, nxt);
            k_cg_pupdate<<<kRedBlocks, BS, 0, I.stream>>>(n, I.scal, nxt, cur, 0, I.cg_z, I.cg_p), ++I.nlaunch;
            std::swap(cur, nxt);
        }
        if (it > I.P.cg_maxit) { *not_conv = 1; it = I.P.cg_maxit; }
        return it;
    }

    // --- PISO ----------------------------------------------------------------
    template <int DIM>
    static int piso_d(Instance &I, void *const *v, double *q, void *const *phi, bool has_st, double vin0, double dt,
                      double *E_out, int *its_out, int *not_conv) {
        GridD g = to_dev(I.g);
        int nb = nblk(g.ncell);
        Fluid<T> fl{(T)I.P.rho1, (T)I.P.rho2, (T)I.P.mu1, (T)I.P.mu2};
        const T *al = tp(I.alpha_new);
        k_rA<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, al, c3(I.phic), fl, (T)dt, tp(I.rA)), ++I.nlaunch;
        void **cf = I.lev[0].c;
        T sig = (T)I.P.sigma;
        int st = has_st ? 1 : 0;
        k_face_coeffs<0, T><<<nblk(I.g.nf[0]), BS, 0, I.stream>>>(g, I.g.nf[0], I.info, tp(I.rA), tp(I.kappa), al, sig,
                                                                 st, tp(cf[0]), tp(I.fst[0])), ++I.nlaunch;
        k_face_coeffs<1, T><<<nblk(I.g.nf[1]), BS, 0, I.stream>>>(g, I.g.nf[1], I.info, tp(I.rA), tp(I.kappa), al, sig,
                                                                 st, tp(cf[1]), tp(I.fst[1])), ++I.nlaunch;
        if (DIM == 3)
            k_face_coeffs<2, T><<<nblk(I.g.nf[2]), BS, 0, I.stream>>>(g, I.g.nf[2], I.info, tp(I.rA), tp(I.kappa), al,
                                                                     sig, st, tp(cf[2]), tp(I.fst[2])), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        int rc = mg_coeffs_d<DIM>(I);
        if (rc) return rc;
        *its_out = 0;
        P3<T> Gp0 = p3(&I.G[0]), Gp1 = p3(&I.G[3]), Gp2 = p3(&I.G[6]);
        C3<T> Gc0 = c3(&I.G[0]), Gc1 = c3(&I.G[3]), Gc2 = c3(&I.G[6]);
        for (int corr = 0; corr < I.P.n_piso; ++corr) {
            k_vel_grad<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, c3(v), (T)vin0, Gp0, Gp1, Gp2), ++I.nlaunch;
            int ps = prof_begin(I, OSCAR_KID_MOMENTUM);
            k_momentum_H<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, c3(v), c3(I.vold), c3(I.phic), al, tp(I.rA), fl,
                                                          (T)vin0, (T)dt, Gc0, Gc1, Gc2, p3(I.hbya)), ++I.nlaunch;
            prof_end(I, ps);
            k_phistar<0, T><<<nblk(I.g.nf[0]), BS, 0, I.stream>>>(g, I.g.nf[0], I.info, tp(I.hbya[0]), tp(I.rA),
                                                                 tp(I.fst[0]), (T)vin0, tp(I.phis[0])), ++I.nlaunch;
            k_phistar<1, T><<<nblk(I.g.nf[1]), BS, 0, I.stream>>>(g, I.g.nf[1], I.info, tp(I.hbya[1]), tp(I.rA),
                                                                 tp(I.fst[1]), T(0), tp(I.phis[1])), ++I.nlaunch;
            if (DIM == 3)
                k_phistar<2, T><<<nblk(I.g.nf[2]), BS, 0, I.stream>>>(g, I.g.nf[2], I.info, tp(I.hbya[2]), tp(I.rA),
                                                                     tp(I.fst[2]), T(0), tp(I.phis[2])), ++I.nlaunch;
            k_rhs<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, c3(I.phis), I.cg_b), ++I.nlaunch;
            OSCAR_LAUNCH_CHECK();
            if (corr == 0) {
                k_sum_field<double><<<kRedBlocks, BS, 0, I.stream>>>(g.ncell, q, 1.0, I.partials), ++I.nlaunch;
                final_sum(I, 0, S_QSUM);
                k_normres<DIM, T><<<kRedBlocks, BS, 0, I.stream>>>(g, I.info, c3(cf), q, I.cg_b, I.scal,
                                                                   1.0 / (double)I.n_fluid, I.partials,
                                                                   I.partials + kRedBlocks), ++I.nlaunch;
                final_sum(I, 0, S_RES);
                final_sum(I, 1, S_NRM);
                OSCAR_LAUNCH_CHECK();
                rc = read_scalars(I);
                if (rc) return rc;
                *E_out = I.scal_host[S_RES] / (I.scal_host[S_NRM] + 1e-20);
            }
            int it = pcg_d<DIM>(I, q, I.cg_b, not_conv);
            if (it < 0) return it;
            *its_out += it;
            k_flux_correct<0, T><<<nblk(I.g.nf[0]), BS, 0, I.stream>>>(g, I.g.nf[0], I.info, tp(I.phis[0]), tp(cf[0]),
                                                                      q, tp(phi[0])), ++I.nlaunch;
            k_flux_correct<1, T><<<nblk(I.g.nf[1]), BS, 0, I.stream>>>(g, I.g.nf[1], I.info, tp(I.phis[1]), tp(cf[1]),
                                                                      q, tp(phi[1])), ++I.nlaunch;
            if (DIM == 3)
                k_flux_correct<2, T><<<nblk(I.g.nf[2]), BS, 0, I.stream>>>(g, I.g.nf[2], I.info, tp(I.phis[2]),
                                                                          tp(cf[2]), q, tp(phi[2])), ++I.nlaunch;
            k_vel_correct<DIM, T><<<nb, BS, 0, I.stream>>>(g, I.info, c3(I.hbya), tp(I.rA), c3(I.fst), q, p3(v)), ++I.nlaunch;
            OSCAR_LAUNCH_CHECK();
        }
        return 0;
    }
    static int piso(Instance &I, void *const *v, double *q, void *const *phi, bool has_st, double vin0, double dt,
                    double *E, int *its, int *not_conv) {
        return I.g.dim == 3 ? piso_d<3>(I, v, q, phi, has_st, vin0, dt, E, its, not_conv)
                            : piso_d<2>(I, v, q, phi, has_st, vin0, dt, E, its, not_conv);
    }

    static int copy_fields(Instance &I, void *const *dst, void *const *src, int nfield_is_face) {
        for (int a = 0; a < I.g.dim; ++a) {
            size_t n = nfield_is_face ? I.g.nf[a] : I.g.ncell;
            if (cudaMemcpyAsync(dst[a], src[a], n * sizeof(T), cudaMemcpyDeviceToDevice, I.stream) != cudaSuccess)
                return OSCAR_E_CUDA;
        }
        return 0;
    }
    static int sum_faces(Instance &I, void *const *a, void *const *b, void *const *out) {
        for (int d = 0; d < I.g.dim; ++d)
            k_sum2<T><<<nblk(I.g.nf[d]), BS, 0, I.stream>>>(I.g.nf[d], tp(a[d]), tp(b[d]), tp(out[d])), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return 0;
    }
    static void swap_alpha(Instance &I) { std::swap(I.alpha, I.alpha_new); }
};

template <typename T> int Solver<T>::setup(Instance &I, const uint8_t *solid_dev, const double *alpha0_dev) {
    GridD g = to_dev(I.g);
    int nb = nblk(g.ncell);
    if (I.g.dim == 3) k_build_info<3><<<nb, BS, 0, I.stream>>>(g, solid_dev, I.info, I.lev[0].fluid), ++I.nlaunch;
    else k_build_info<2><<<nb, BS, 0, I.stream>>>(g, solid_dev, I.info, I.lev[0].fluid), ++I.nlaunch;
    k_load_alpha<T><<<nb, BS, 0, I.stream>>>(g.ncell, I.info, alpha0_dev, (T *)I.alpha), ++I.nlaunch;
    for (int l = 1; l < I.nlev; ++l) {
        Level &F = I.lev[l - 1], &L = I.lev[l];
        k_mg_fluid_coarsen<<<nblk(L.g.ncell), BS, 0, I.stream>>>(to_dev(F.g), to_dev(L.g), F.r[0], F.r[1], F.r[2],
                                                                 F.fluid, L.fluid), ++I.nlaunch;
    }
    OSCAR_LAUNCH_CHECK();
    return Impl<T>::interface_(I, I.alpha);
}

// Section 3.1: viscous-drag step
template <typename T> int Solver<T>::drag_step(Instance &I, double dt) {
    using X = Impl<T>;
    int rc = X::transport(I, I.phi_vd, dt);
    if (rc) return rc;
    if ((rc = X::sum_faces(I, I.phi_vd, I.phi_cr, I.phic))) return rc;
    if ((rc = X::copy_fields(I, I.vold, I.u_vd, 0))) return rc;
    double E = 0.0;
    int its = 0, nc = 0;
    rc = X::piso(I, I.u_vd, I.p_vd, I.phi_vd, false, I.P.U_inlet, dt, &E, &its, &nc);
    if (rc) return rc;
    X::swap_alpha(I);
    if ((rc = X::interface_(I, I.alpha))) return rc;
    I.cg_iters_last = its;
    I.cg_iters_total += its;
    I.cell_updates += I.n_fluid;
    return nc ? OSCAR_E_NOT_CONVERGED : 0;
}

// Section 3.2: capillary-relaxation sub-steps with the early exit and the
// reconstruction u = u_vd + (1/N) sum_k u_cr^{n,k}
template <typename T> int Solver<T>::relax(Instance &I, double dt, int N, int *kf_out, double *test_out) {
    using X = Impl<T>;
    int rc;
    for (int a = 0; a < I.g.dim; ++a)
        if (cudaMemsetAsync(I.u_sum[a], 0, I.g.ncell * sizeof(double), I.stream) != cudaSuccess) return OSCAR_E_CUDA;
    int kf = 0, nc_any = 0;
    double test = 0.0;
    for (int k = 0; k < N; ++k) {
        if ((rc = X::transport(I, I.phi_cr, dt))) return rc;
        if ((rc = X::interface_(I, I.alpha_new))) return rc;
        if ((rc = X::sum_faces(I, I.phi_vd, I.phi_cr, I.phic))) return rc;
        if ((rc = X::copy_fields(I, I.vold, I.u_cr, 0))) return rc;
        double E = 0.0;
        int its = 0, nc = 0;
        rc = X::piso(I, I.u_cr, I.p_cr, I.phi_cr, true, 0.0, dt, &E, &its, &nc);
        if (rc) return rc;
        nc_any |= nc;
        X::swap_alpha(I);
        P3<double> us;
        for (int a = 0; a < 3; ++a) us.a[a] = I.u_sum[a];
        if (I.g.dim == 3)
            k_relax_accum<3, T><<<kRedBlocks, BS, 0, I.stream>>>(I.g.ncell, I.info, X::c3(I.u_cr), X::c3(I.vold), us,
                                                                 I.partials), ++I.nlaunch;
        else
            k_relax_accum<2, T><<<kRedBlocks, BS, 0, I.stream>>>(I.g.ncell, I.info, X::c3(I.u_cr), X::c3(I.vold), us,
                                                                 I.partials), ++I.nlaunch;
        X::final_sum(I, 0, S_DUMAX, true);
        OSCAR_LAUNCH_CHECK();
        if ((rc = X::read_scalars(I))) return rc;
        double dU = I.scal_host[S_DUMAX] / I.P.U_inlet;
        I.last_E = E;
        I.last_dU = dU;
        I.cg_iters_last = its;
        I.cg_iters_total += its;
        I.cell_updates += I.n_fluid;
        kf = k + 1;
        test = (I.P.conv_mode == OSCAR_CONV_DU_MAX) ? dU : E;
        if (!isfinite(test)) return OSCAR_E_NAN;
        if (test < I.P.conv_tol) break;
    }
    I.last_kf = kf;
    I.last_N = N;
    if (kf_out) *kf_out = kf;
    if (test_out) *test_out = test;
    return nc_any ? OSCAR_E_NOT_CONVERGED : 0;
}

// Section 2.2: standard time-stepping
template <typename T> int Solver<T>::standard_step(Instance &I, double dt) {
    using X = Impl<T>;
    int rc = X::transport(I, I.phi_vd, dt);
    if (rc) return rc;
    if ((rc = X::interface_(I, I.alpha_new))) return rc;
    if ((rc = X::copy_fields(I, I.phic, I.phi_vd, 1))) return rc;
    if ((rc = X::copy_fields(I, I.vold, I.u_vd, 0))) return rc;
    double E = 0.0;
    int its = 0, nc = 0;
    rc = X::piso(I, I.u_vd, I.p_vd, I.phi_vd, true, I.P.U_inlet, dt, &E, &its, &nc);
    if (rc) return rc;
    X::swap_alpha(I);
    for (int a = 0; a < I.g.dim; ++a)
        if (cudaMemsetAsync(I.u_sum[a], 0, I.g.ncell * sizeof(double), I.stream) != cudaSuccess) return OSCAR_E_CUDA;
    I.last_E = E;
    I.last_N = 1;
    I.cg_iters_last = its;
    I.cg_iters_total += its;
    I.cell_updates += I.n_fluid;
    return nc ? OSCAR_E_NOT_CONVERGED : 0;
}

template <typename T>
__global__ void k_report_u(int n, const T *__restrict__ uvd, const double *__restrict__ usum, double invN,
                           double *__restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = (double)uvd[c] + usum[c] * invN;
}
static __global__ void k_add_pd(int n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = a[c] + b[c];
}

template <typename T> int Solver<T>::field_to_device(Instance &I, int which, double *dst, size_t n) {
    int nc = I.g.ncell;
    cudaStream_t s = I.stream;
    auto cvt = [&](const void *src, size_t len) { k_convert<T, double><<<nblk(len), BS, 0, s>>>((int)len, (const T *)src, dst), ++I.nlaunch; };
    if (which == OSCAR_FIELD_ALPHA) cvt(I.alpha, nc);
    else if (which == OSCAR_FIELD_P) k_add_pd<<<nblk(nc), BS, 0, s>>>(nc, I.p_vd, I.p_cr, dst), ++I.nlaunch;
    else if (which >= 2 && which <= 4) {
        int a = which - 2;
        if (a >= I.g.dim) cudaMemsetAsync(dst, 0, n * sizeof(double), s);
        else k_report_u<T><<<nblk(nc), BS, 0, s>>>(nc, (const T *)I.u_vd[a], I.u_sum[a], 1.0 / (double)I.last_N, dst), ++I.nlaunch;
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
    int nc = I.g.ncell;
    cudaStream_t s = I.stream;
    auto cvt = [&](void *dst, size_t len) { k_convert<double, T><<<nblk(len), BS, 0, s>>>((int)len, src, (T *)dst), ++I.nlaunch; };
    if (which == OSCAR_FIELD_ALPHA) {
        k_load_alpha<T><<<nblk(nc), BS, 0, s>>>(nc, I.info, src, (T *)I.alpha), ++I.nlaunch;
        OSCAR_LAUNCH_CHECK();
        return Impl<T>::interface_(I, I.alpha);
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
    k_sum_field<T><<<kRedBlocks, BS, 0, I.stream>>>(I.g.ncell, (const T *)I.alpha, I.g.V, I.partials), ++I.nlaunch;
    Impl<T>::final_sum(I, 0, S_VOL);
    OSCAR_LAUNCH_CHECK();
    int rc = Impl<T>::read_scalars(I);
    if (rc) return rc;
    *out = I.scal_host[S_VOL];
    return 0;
}

}  // namespace oscar
