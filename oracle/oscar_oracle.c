/*
 * OSCAR oracle: a plain, slow, single-threaded FP64 CPU implementation of the
 * capillary-relaxation / viscous-drag time stepping of Maes & Menke,
 * "OSCAR: Operator Splitting with Capillary Relaxation" (arXiv 2105.10576).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load this library. It shares no code, header or
 * constant with the CUDA path. Every loop below visits cells and faces in the
 * plain order; there is no blocking, fusion or reordering.
 *
 * Grid model: uniform Cartesian cells (x fastest), per-cell solid mask. Faces of
 * direction a are stored per direction; the face on the low side of cell
 * (i,j,k) in direction a has index face_index(a,i,j,k); fluxes are oriented +a.
 * x-min is the inlet, x-max the outlet, every other boundary and every
 * fluid/solid face is a wall (Section 3, problem statement).
 *
 * Paper references (section / equation):
 *   mixture properties      Section 2.1 (rho, mu single-field; mu printed as rho, read as mu)
 *   momentum + continuity   Eqs. NSEVOF1/NSEVOF2; drag Eqs. NSE1d/md; relaxation Eqs. NSEc/mc
 *   alpha transport         Eqs. phaseEq/alphaExp (explicit Euler); drag Eq. VOFd; relaxation Eq. VOFc;
 *                           vanLeer + interface compression (Section 4, Implementation)
 *   CSF, normal, curvature  Section 2.1 (f_st = sigma kappa grad alpha, n = grad alpha/|grad alpha|)
 *   contact angle           boundary conditions of Eqs. VOFd/VOFc (n . n_wall = cos theta)
 *   PISO (3 correctors)     Section 2.2 (u* = (H+f)/A; div(1/A grad p) = div u*; u = u* - 1/A grad p)
 *   CFL, Brackbill limits   Section 2.2
 *   additive / sequential splitting, residual E_k, reconstruction: Section 3, 3.1, 3.2
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_F_NONE 0
#define OR_F_INTERIOR 1
#define OR_F_WALL 2
#define OR_F_INLET 3
#define OR_F_OUTLET 4

#define OR_CONV_PRES_RESID 0
#define OR_CONV_DU_MAX 1
#define OR_CONV_AREA 2

/* exact (banded Cholesky) pressure solves up to this many multiply-adds */
#define OR_BANDED_MAX_WORK 4.0e8

typedef struct {
    int dim, nx, ny, nz;
    double hx, hy, hz;
    double rho1, rho2, mu1, mu2, sigma, theta_deg;
    double U_inlet, alpha_inlet;
    int n_piso, n_smooth;
    double c_alpha;
    int conv_mode;
    double conv_tol;
    double cg_rtol;
    int cg_maxit;
    int precision; /* ignored: the oracle is FP64 throughout */
} or_params;

typedef struct {
    int dim;
    int n[3];
    double h[3];
    int ncell;
    int nface[3];
    double V;      /* cell volume (area in 2D) */
    double S[3];   /* face area per direction (length in 2D) */
    const uint8_t *solid;
} or_grid;

typedef struct {
    or_params P;
    or_grid g;
    uint8_t *solid;
    double *alpha, *kappa, *alpha_s;
    double *nf[3];
    double *u_vd[3], *u_cr[3], *u_cr_sum[3];
    double *p_vd, *p_cr;
    double *phi_vd[3], *phi_cr[3];
    /* statistics of the last call */
    double last_E, last_dU;
    int last_kf, last_N;
    long cg_iters_total;
    int cg_iters_last, cg_fail;
} or_state;

/* ------------------------------------------------------------------------- */
/* grid helpers                                                               */
/* ------------------------------------------------------------------------- */
static void grid_init(or_grid *g, const or_params *P, const uint8_t *solid) {
    g->dim = P->dim;
    g->n[0] = P->nx; g->n[1] = P->ny; g->n[2] = (P->dim == 3) ? P->nz : 1;
    g->h[0] = P->hx; g->h[1] = P->hy; g->h[2] = P->hz;
    g->ncell = g->n[0] * g->n[1] * g->n[2];
    g->nface[0] = (g->n[0] + 1) * g->n[1] * g->n[2];
    g->nface[1] = g->n[0] * (g->n[1] + 1) * g->n[2];
    g->nface[2] = g->n[0] * g->n[1] * (g->n[2] + 1);
    g->V = 1.0;
    for (int a = 0; a < g->dim; ++a) g->V *= g->h[a];
    for (int a = 0; a < 3; ++a) g->S[a] = (a < g->dim) ? g->V / g->h[a] : 0.0;
    g->solid = solid;
}

static int cidx(const or_grid *g, int i, int j, int k) { return i + g->n[0] * (j + g->n[1] * k); }

static int fidx(const or_grid *g, int a, int i, int j, int k) {
    if (a == 0) return i + (g->n[0] + 1) * (j + g->n[1] * k);
    if (a == 1) return i + g->n[0] * (j + (g->n[1] + 1) * k);
    return i + g->n[0] * (j + g->n[1] * k);
}

static void cijk(const or_grid *g, int c, int *ijk) {
    ijk[0] = c % g->n[0];
    ijk[1] = (c / g->n[0]) % g->n[1];
    ijk[2] = c / (g->n[0] * g->n[1]);
}

static int is_fluid(const or_grid *g, const int *ijk) {
    for (int a = 0; a < 3; ++a)
        if (ijk[a] < 0 || ijk[a] >= g->n[a]) return 0;
    return g->solid[cidx(g, ijk[0], ijk[1], ijk[2])] == 0;
}

/* Face f of direction a at face coordinates (i,j,k) (i.e. low side of cell ijk).
 * Sets *L, *H to the fluid cell indices on each side (-1 if absent) and returns
 * the face type. */
static int face_cells(const or_grid *g, int a, const int *fijk, int *L, int *H) {
    int lo[3] = {fijk[0], fijk[1], fijk[2]};
    int hi[3] = {fijk[0], fijk[1], fijk[2]};
    lo[a] -= 1;
    int lin = lo[a] >= 0, hin = hi[a] < g->n[a];
    int lf = lin && is_fluid(g, lo), hf = hin && is_fluid(g, hi);
    *L = lf ? cidx(g, lo[0], lo[1], lo[2]) : -1;
    *H = hf ? cidx(g, hi[0], hi[1], hi[2]) : -1;
    if (lf && hf) return OR_F_INTERIOR;
    if (!lf && !hf) return OR_F_NONE;
    if (lf) { /* fluid on the low side */
        if (!hin) return a == 0 ? OR_F_OUTLET : OR_F_WALL;
        return OR_F_WALL;
    }
    if (!lin) return a == 0 ? OR_F_INLET : OR_F_WALL;
    return OR_F_WALL;
}

/* Face of cell c in direction a on side s (0 low, 1 high): face index, type,
 * neighbour (or -1). */
static int cell_face(const or_grid *g, int c, int a, int s, int *f, int *nb) {
    int ijk[3];
    cijk(g, c, ijk);
    int fijk[3] = {ijk[0], ijk[1], ijk[2]};
    if (s) fijk[a] += 1;
    *f = fidx(g, a, fijk[0], fijk[1], fijk[2]);
    int L, H;
    int t = face_cells(g, a, fijk, &L, &H);
    *nb = s ? H : L;
    return t;
}

/* Iterate faces of direction a: call face_cells on every face coordinate. */
#define FOR_FACES(g, a, fijk, f)                                                   \
    for (int _k = 0; _k < (g)->n[2] + ((a) == 2); ++_k)                             \
        for (int _j = 0; _j < (g)->n[1] + ((a) == 1); ++_j)                         \
            for (int _i = 0; _i < (g)->n[0] + ((a) == 0); ++_i)                     \
                for (int fijk[3] = {_i, _j, _k}, f = fidx(g, a, _i, _j, _k), _once = 1; \
                     _once; _once = 0)

/* ------------------------------------------------------------------------- */
/* Section 2.1: single-field mixture properties                              */
/* ------------------------------------------------------------------------- */
static double mix_rho(const or_params *P, double al) { return al * P->rho1 + (1.0 - al) * P->rho2; }
static double mix_mu(const or_params *P, double al) { return al * P->mu1 + (1.0 - al) * P->mu2; }

/* ------------------------------------------------------------------------- */
/* Section 2.2: CFL and Brackbill limits; Section 3.2: N sub-steps            */
/* out[0]=dt_cfl, out[1]=dt_B, out[2]=dt_vd, out[3]=N                         */
/*                                                                           */
/* The CFL limit is Delta x / u with u the flow velocity. For a constant time */
/* step fixed before the run, u is taken as the largest cross-section mean of */
/* the x velocity that mass conservation fixes: the injected flux U A_in      */
/* passes every cross-section x = const, so its mean speed there is           */
/* U A_in / A(x), largest at the narrowest section. A(x) counts the fluid     */
/* cells of column i (all j, k). solid = NULL is an open channel (u = U).     */
/* Returns -1 when some column has no fluid cell while the inlet has one (no  */
/* path from the inlet to the outlet), else 0.                                */
/* ------------------------------------------------------------------------- */
int or_timesteps(const or_params *P, const uint8_t *solid, double c_cfl, double *out) {
    double hmin = P->hx;
    if (P->hy < hmin) hmin = P->hy;
    if (P->dim == 3 && P->hz < hmin) hmin = P->hz;
    double u = P->U_inlet;
    if (solid) {
        int nz = P->dim == 3 ? P->nz : 1;
        long a_in = -1, a_min = -1;
        for (int i = 0; i < P->nx; ++i) {
            long a = 0;
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < P->ny; ++j)
                    if (solid[i + P->nx * (j + P->ny * k)] == 0) a += 1;
            if (i == 0) a_in = a;
            if (a_min < 0 || a < a_min) a_min = a;
        }
        if (a_in > 0) {
            if (a_min == 0) return -1;
            u = P->U_inlet * (double)a_in / (double)a_min;
        }
    }
    double dt_cfl = P->hx / u;                           /* Delta x / u, flow along x */
    double rho_bar = 0.5 * (P->rho1 + P->rho2);          /* average density of the two phases */
    double dt_b = sqrt(rho_bar * hmin * hmin * hmin / (2.0 * M_PI * P->sigma));
    double dt_vd = c_cfl * dt_cfl;
    double N = floor(dt_vd / dt_b) + 1.0;                /* smallest integer with dt_vd/N < dt_B */
    out[0] = dt_cfl; out[1] = dt_b; out[2] = dt_vd; out[3] = N;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* alpha transport, Eq. alphaExp with a vanLeer high-order flux, interface   */
/* compression and a Zalesak flux-corrected-transport limiter                 */
/* ------------------------------------------------------------------------- */

/* vanLeer face value, psi(r) = (r+|r|)/(1+|r|), alpha_f = aU + psi/2 (aD - aU),
 * r = (aU - aUU)/(aD - aU); for r > 0 this equals aU + du*dc/(du+dc). */
static double vanleer_face(double aUU, int hasUU, double aU, double aD) {
    double dc = aD - aU;
    double du = hasUU ? (aU - aUU) : 0.0;
    if (du * dc > 0.0) return aU + du * dc / (du + dc);
    return aU;
}

/* Compute, for every face of direction a, the low-order (upwind) flux FL and the
 * antidiffusive flux AD = F_high - F_low. */
static void transport_face_fluxes(const or_grid *g, const double *alpha, double *const phi[3],
                                  double *const nf[3], double c_alpha, double alpha_in,
                                  double *FL[3], double *AD[3]) {
    for (int a = 0; a < g->dim; ++a) {
        FOR_FACES(g, a, fijk, f) {
            int L, H;
            int t = face_cells(g, a, fijk, &L, &H);
            double ph = phi[a][f];
            FL[a][f] = 0.0;
            AD[a][f] = 0.0;
            if (t == OR_F_INTERIOR) {
                int U, D, UU = -1;
                int uu[3] = {fijk[0], fijk[1], fijk[2]};
                if (ph >= 0.0) { U = L; D = H; uu[a] -= 2; }
                else { U = H; D = L; uu[a] += 1; }
                if (is_fluid(g, uu)) UU = cidx(g, uu[0], uu[1], uu[2]);
                double aU = alpha[U], aD = alpha[D];
                double aUU = UU >= 0 ? alpha[UU] : 0.0;
                double a_vl = vanleer_face(aUU, UU >= 0, aU, aD);
                double flow = ph * aU;
                /* compression velocity flux phi_r = c_alpha |phi| n_f (face-normal part of n) */
                double phir = c_alpha * fabs(ph) * nf[a][f];
                double fc;
                if (phir >= 0.0) fc = phir * alpha[L] * (1.0 - alpha[H]);
                else fc = phir * alpha[H] * (1.0 - alpha[L]);
                double fhigh = ph * a_vl + fc;
                FL[a][f] = flow;
                AD[a][f] = fhigh - flow;
            } else if (t == OR_F_INLET) {
                FL[a][f] = ph >= 0.0 ? ph * alpha_in : ph * alpha[H];
            } else if (t == OR_F_OUTLET) {
                FL[a][f] = ph * alpha[L];
            }
        }
    }
}

/* alpha_new = alpha - dt/V sum_f outward flux, limited (Zalesak 1979). */
void or_transport(const or_grid *g, const double *alpha, double *const phi[3], double *const nf[3],
                  double dt, double c_alpha, double alpha_in, double *alpha_new) {
    int nc = g->ncell;
    double *FL[3] = {0}, *AD[3] = {0}, *LAM[3] = {0};
    for (int a = 0; a < g->dim; ++a) {
        FL[a] = calloc(g->nface[a], sizeof(double));
        AD[a] = calloc(g->nface[a], sizeof(double));
        LAM[a] = calloc(g->nface[a], sizeof(double));
    }
    transport_face_fluxes(g, alpha, phi, nf, c_alpha, alpha_in, FL, AD);
    double *aL = calloc(nc, sizeof(double));
    double *Rp = calloc(nc, sizeof(double));
    double *Rm = calloc(nc, sizeof(double));
    double rV = dt / g->V;
    /* low-order solution */
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) continue;
        double out = 0.0;
        for (int a = 0; a < g->dim; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                cell_face(g, c, a, s, &f, &nb);
                out += s ? FL[a][f] : -FL[a][f];
            }
        aL[c] = alpha[c] - rV * out;
    }
    /* local bounds and Zalesak ratios */
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) continue;
        double amax = alpha[c] > aL[c] ? alpha[c] : aL[c];
        double amin = alpha[c] < aL[c] ? alpha[c] : aL[c];
        double Pp = 0.0, Pm = 0.0;
        for (int a = 0; a < g->dim; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                int t = cell_face(g, c, a, s, &f, &nb);
                if (t == OR_F_INTERIOR) {
                    if (alpha[nb] > amax) amax = alpha[nb];
                    if (aL[nb] > amax) amax = aL[nb];
                    if (alpha[nb] < amin) amin = alpha[nb];
                    if (aL[nb] < amin) amin = aL[nb];
                }
                double aout = s ? AD[a][f] : -AD[a][f];
                if (aout > 0.0) Pm += aout; else Pp += -aout;
            }
        if (amax > 1.0) amax = 1.0;
        if (amin < 0.0) amin = 0.0;
        double Qp = (amax - aL[c]) / rV;
        double Qm = (aL[c] - amin) / rV;
        if (Qp < 0.0) Qp = 0.0;
        if (Qm < 0.0) Qm = 0.0;
        Rp[c] = Pp > 0.0 ? (Qp / Pp < 1.0 ? Qp / Pp : 1.0) : 0.0;
        Rm[c] = Pm > 0.0 ? (Qm / Pm < 1.0 ? Qm / Pm : 1.0) : 0.0;
    }
    /* face limiter lambda_f */
    for (int a = 0; a < g->dim; ++a) {
        FOR_FACES(g, a, fijk, f) {
            int L, H;
            int t = face_cells(g, a, fijk, &L, &H);
            if (t != OR_F_INTERIOR) continue;
            double l;
            if (AD[a][f] >= 0.0) l = Rm[L] < Rp[H] ? Rm[L] : Rp[H];
            else l = Rm[H] < Rp[L] ? Rm[H] : Rp[L];
            LAM[a][f] = l;
        }
    }
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) { alpha_new[c] = 0.0; continue; }
        double out = 0.0;
        for (int a = 0; a < g->dim; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                cell_face(g, c, a, s, &f, &nb);
                double fl = LAM[a][f] * AD[a][f];
                out += s ? fl : -fl;
            }
        alpha_new[c] = aL[c] - rV * out;
    }
    free(aL); free(Rp); free(Rm);
    for (int a = 0; a < g->dim; ++a) { free(FL[a]); free(AD[a]); free(LAM[a]); }
}

/* ------------------------------------------------------------------------- */
/* Section 2.1: interface normal, curvature; contact angle at walls           */
/* ------------------------------------------------------------------------- */
/* Gauss gradient along b of a cell field with zero-gradient boundary faces. */
static double gauss_grad_scalar(const or_grid *g, const double *x, int c, int b) {
    double fv[2];
    for (int s = 0; s < 2; ++s) {
        int f, nb;
        int t = cell_face(g, c, b, s, &f, &nb);
        fv[s] = (t == OR_F_INTERIOR) ? 0.5 * (x[c] + x[nb]) : x[c];
    }
    return (fv[1] - fv[0]) / g->h[b];
}

/* alpha_s: n_smooth passes of face-area-weighted averages of linearly
 * interpolated face values; nf: face-normal component of n = g/(|g|+delta_N)
 * with the contact angle imposed at walls; kappa = -div(n). */
void or_interface(const or_grid *g, const double *alpha, int n_smooth, double theta_deg,
                  double *alpha_s, double *nf[3], double *kappa) {
    int nc = g->ncell;
    double *tmp = calloc(nc, sizeof(double));
    for (int c = 0; c < nc; ++c) alpha_s[c] = g->solid[c] ? 0.0 : alpha[c];
    for (int pass = 0; pass < n_smooth; ++pass) {
        for (int c = 0; c < nc; ++c) {
            if (g->solid[c]) { tmp[c] = 0.0; continue; }
            double num = 0.0, den = 0.0;
            for (int a = 0; a < g->dim; ++a)
                for (int s = 0; s < 2; ++s) {
                    int f, nb;
                    int t = cell_face(g, c, a, s, &f, &nb);
                    double af = (t == OR_F_INTERIOR) ? 0.5 * (alpha_s[c] + alpha_s[nb]) : alpha_s[c];
                    num += af * g->S[a];
                    den += g->S[a];
                }
            tmp[c] = num / den;
        }
        memcpy(alpha_s, tmp, nc * sizeof(double));
    }
    double hbar = pow(g->V, 1.0 / g->dim);
    double deltaN = 1e-8 / hbar;
    double ct = cos(theta_deg * M_PI / 180.0);
    for (int a = 0; a < g->dim; ++a) {
        FOR_FACES(g, a, fijk, f) {
            int L, H;
            int t = face_cells(g, a, fijk, &L, &H);
            double n = 0.0;
            if (t == OR_F_INTERIOR) {
                double gv[3] = {0, 0, 0};
                gv[a] = (alpha_s[H] - alpha_s[L]) / g->h[a];
                for (int b = 0; b < g->dim; ++b) {
                    if (b == a) continue;
                    gv[b] = 0.5 * (gauss_grad_scalar(g, alpha_s, L, b) + gauss_grad_scalar(g, alpha_s, H, b));
                }
                double mag = 0.0;
                for (int b = 0; b < g->dim; ++b) mag += gv[b] * gv[b];
                mag = sqrt(mag);
                n = gv[a] / (mag + deltaN);
            } else if (t == OR_F_WALL) {
                /* n . n_wall = cos(theta), n_wall pointing out of the fluid cell */
                n = (L >= 0) ? ct : -ct;
            }
            nf[a][f] = n;
        }
    }
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) { kappa[c] = 0.0; continue; }
        double k = 0.0;
        for (int a = 0; a < g->dim; ++a) {
            int f0, f1, nb;
            cell_face(g, c, a, 0, &f0, &nb);
            cell_face(g, c, a, 1, &f1, &nb);
            k += (nf[a][f1] - nf[a][f0]) / g->h[a];
        }
        kappa[c] = -k;
    }
    free(tmp);
}

/* ------------------------------------------------------------------------- */
/* Pressure equation: div(1/A grad p) = div(phi*) as an SPD system M q = b    */
/* (M q)_P = sum_f c_f (q_P - q_N) + sum_outlet c_f q_P                       */
/* ------------------------------------------------------------------------- */
void or_poisson_apply(const or_grid *g, double *const cf[3], const double *q, double *y) {
    for (int c = 0; c < g->ncell; ++c) {
        if (g->solid[c]) { y[c] = 0.0; continue; }
        double acc = 0.0;
        for (int a = 0; a < g->dim; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                int t = cell_face(g, c, a, s, &f, &nb);
                if (t == OR_F_INTERIOR) acc += cf[a][f] * (q[c] - q[nb]);
                else if (t == OR_F_OUTLET) acc += cf[a][f] * q[c];
            }
        y[c] = acc;
    }
}

static void poisson_diag(const or_grid *g, double *const cf[3], double *d) {
    for (int c = 0; c < g->ncell; ++c) {
        double acc = 0.0;
        if (!g->solid[c])
            for (int a = 0; a < g->dim; ++a)
                for (int s = 0; s < 2; ++s) {
                    int f, nb;
                    int t = cell_face(g, c, a, s, &f, &nb);
                    if (t == OR_F_INTERIOR || t == OR_F_OUTLET) acc += cf[a][f];
                }
        d[c] = acc;
    }
}

static double dot_fluid(const or_grid *g, const double *x, const double *y) {
    double s = 0.0;
    for (int c = 0; c < g->ncell; ++c)
        if (!g->solid[c]) s += x[c] * y[c];
    return s;
}

/* Jacobi-preconditioned conjugate gradients; stops when the recursively
 * updated residual satisfies ||r||_2 <= rtol * ||b||_2 (rtol * ||r0||_2 if
 * b = 0). Returns iterations (negative if maxit was reached). */
int or_poisson_cg(const or_grid *g, double *const cf[3], const double *b, double *q,
                  double rtol, int maxit) {
    int nc = g->ncell;
    double *r = calloc(nc, sizeof(double)), *z = calloc(nc, sizeof(double));
    double *p = calloc(nc, sizeof(double)), *Ap = calloc(nc, sizeof(double));
    double *d = calloc(nc, sizeof(double));
    poisson_diag(g, cf, d);
    or_poisson_apply(g, cf, q, Ap);
    for (int c = 0; c < nc; ++c) r[c] = g->solid[c] ? 0.0 : b[c] - Ap[c];
    double bn = sqrt(dot_fluid(g, b, b));
    double rn = sqrt(dot_fluid(g, r, r));
    double target = rtol * (bn > 0.0 ? bn : rn);
    int it = 0;
    if (rn > target) {
        for (int c = 0; c < nc; ++c) z[c] = g->solid[c] ? 0.0 : r[c] / d[c];
        memcpy(p, z, nc * sizeof(double));
        double rz = dot_fluid(g, r, z);
        for (it = 1; it <= maxit; ++it) {
            or_poisson_apply(g, cf, p, Ap);
            double pAp = dot_fluid(g, p, Ap);
            double al = rz / pAp;
            for (int c = 0; c < nc; ++c) {
                if (g->solid[c]) continue;
                q[c] += al * p[c];
                r[c] -= al * Ap[c];
            }
            rn = sqrt(dot_fluid(g, r, r));
            if (rn <= target) break;
            for (int c = 0; c < nc; ++c) z[c] = g->solid[c] ? 0.0 : r[c] / d[c];
            double rz1 = dot_fluid(g, r, z);
            double be = rz1 / rz;
            rz = rz1;
            for (int c = 0; c < nc; ++c) p[c] = g->solid[c] ? 0.0 : z[c] + be * p[c];
        }
        if (it > maxit) it = -maxit;
    }
    free(r); free(z); free(p); free(Ap); free(d);
    return it;
}

/* Dense Cholesky solve of M q = b over fluid cells (tiny grids only). */
int or_poisson_dense(const or_grid *g, double *const cf[3], const double *b, double *q) {
    int nc = g->ncell, m = 0;
    int *map = malloc(nc * sizeof(int));
    for (int c = 0; c < nc; ++c) map[c] = g->solid[c] ? -1 : m++;
    double *A = calloc((size_t)m * m, sizeof(double));
    double *e = calloc(nc, sizeof(double)), *col = calloc(nc, sizeof(double));
    for (int c = 0; c < nc; ++c) {
        if (map[c] < 0) continue;
        memset(e, 0, nc * sizeof(double));
        e[c] = 1.0;
        or_poisson_apply(g, cf, e, col);
        for (int r = 0; r < nc; ++r)
            if (map[r] >= 0) A[(size_t)map[r] * m + map[c]] = col[r];
    }
    /* in-place Cholesky, lower triangle */
    for (int j = 0; j < m; ++j) {
        double s = A[(size_t)j * m + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * m + k] * A[(size_t)j * m + k];
        if (s <= 0.0) { free(map); free(A); free(e); free(col); return -1; }
        double ljj = sqrt(s);
        A[(size_t)j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double t = A[(size_t)i * m + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * m + k] * A[(size_t)j * m + k];
            A[(size_t)i * m + j] = t / ljj;
        }
    }
    double *y = calloc(m, sizeof(double));
    for (int c = 0; c < nc; ++c) if (map[c] >= 0) y[map[c]] = b[c];
    for (int i = 0; i < m; ++i) {
        double t = y[i];
        for (int k = 0; k < i; ++k) t -= A[(size_t)i * m + k] * y[k];
        y[i] = t / A[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < m; ++k) t -= A[(size_t)k * m + i] * y[k];
        y[i] = t / A[(size_t)i * m + i];
    }
    for (int c = 0; c < nc; ++c) q[c] = map[c] >= 0 ? y[map[c]] : 0.0;
    free(map); free(A); free(e); free(col); free(y);
    return 0;
}

/* Banded Cholesky solve of M q = b over fluid cells: the exact solution of
 * the pressure equation up to rounding. Cells are numbered with the shortest
 * axis fastest so the bandwidth is the product of the two shortest extents.
 * Returns -1 if M is not positive definite, -2 if the band is too wide
 * (more than max_work multiply-adds). */
int or_poisson_banded(const or_grid *g, double *const cf[3], const double *b, double *q, double max_work) {
    int nc = g->ncell;
    int ax[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)   /* sort axes by extent, shortest first (x wins ties) */
        for (int j = i + 1; j < 3; ++j)
            if (g->n[ax[j]] < g->n[ax[i]]) { int t = ax[i]; ax[i] = ax[j]; ax[j] = t; }
    int *map = malloc(nc * sizeof(int));
    int m = 0;
    int ijk[3];
    for (int s2 = 0; s2 < g->n[ax[2]]; ++s2)
        for (int s1 = 0; s1 < g->n[ax[1]]; ++s1)
            for (int s0 = 0; s0 < g->n[ax[0]]; ++s0) {
                ijk[ax[0]] = s0; ijk[ax[1]] = s1; ijk[ax[2]] = s2;
                int c = cidx(g, ijk[0], ijk[1], ijk[2]);
                map[c] = g->solid[c] ? -1 : m++;
            }
    /* bandwidth over the couplings of the operator */
    int bw = 0;
    for (int c = 0; c < nc; ++c) {
        if (map[c] < 0) continue;
        for (int a = 0; a < g->dim; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                if (cell_face(g, c, a, s, &f, &nb) == OR_F_INTERIOR) {
                    int d = map[c] > map[nb] ? map[c] - map[nb] : map[nb] - map[c];
                    if (d > bw) bw = d;
                }
            }
    }
    if ((double)m * (bw + 1) * (bw + 1) > max_work) { free(map); return -2; }
    int W = bw + 1;   /* row r holds A(r, r-d) at L[r*W + d] */
    double *L = calloc((size_t)m * W, sizeof(double));
    for (int c = 0; c < nc; ++c) {
        int r = map[c];
        if (r < 0) continue;
        double diag = 0.0;
        for (int a = 0; a < g->dim; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                int t = cell_face(g, c, a, s, &f, &nb);
                if (t == OR_F_INTERIOR) {
                    diag += cf[a][f];
                    int rn = map[nb];
                    if (rn < r) L[(size_t)r * W + (r - rn)] -= cf[a][f];
                } else if (t == OR_F_OUTLET) {
                    diag += cf[a][f];
                }
            }
        L[(size_t)r * W] = diag;
    }
    /* in-place band Cholesky: A = L L^T */
    for (int j = 0; j < m; ++j) {
        double sum = L[(size_t)j * W];
        int k0 = j - bw > 0 ? j - bw : 0;
        for (int k = k0; k < j; ++k) {
            double ljk = L[(size_t)j * W + (j - k)];
            sum -= ljk * ljk;
        }
        if (sum <= 0.0) { free(map); free(L); return -1; }
        double ljj = sqrt(sum);
        L[(size_t)j * W] = ljj;
        int i1 = j + bw < m - 1 ? j + bw : m - 1;
        for (int i = j + 1; i <= i1; ++i) {
            double t = L[(size_t)i * W + (i - j)];
            int kk0 = i - bw > k0 ? i - bw : k0;
            for (int k = kk0; k < j; ++k) t -= L[(size_t)i * W + (i - k)] * L[(size_t)j * W + (j - k)];
            L[(size_t)i * W + (i - j)] = t / ljj;
        }
    }
    double *y = calloc(m, sizeof(double));
    for (int c = 0; c < nc; ++c) if (map[c] >= 0) y[map[c]] = b[c];
    for (int i = 0; i < m; ++i) {   /* L y' = y */
        double t = y[i];
        int k0 = i - bw > 0 ? i - bw : 0;
        for (int k = k0; k < i; ++k) t -= L[(size_t)i * W + (i - k)] * y[k];
        y[i] = t / L[(size_t)i * W];
    }
    for (int i = m - 1; i >= 0; --i) {   /* L^T q = y' */
        double t = y[i];
        int k1 = i + bw < m - 1 ? i + bw : m - 1;
        for (int k = i + 1; k <= k1; ++k) t -= L[(size_t)k * W + (k - i)] * y[k];
        y[i] = t / L[(size_t)i * W];
    }
    for (int c = 0; c < nc; ++c) q[c] = map[c] >= 0 ? y[map[c]] : 0.0;
    free(map); free(L); free(y);
    return 0;
}

/* Normalised L1 residual of M q = b: sum|b - Mq| / (sum|Mq - M qbar| + sum|b - M qbar| + 1e-20),
 * qbar the mean of q over fluid cells (the normalised residual norm of Section 3.2). */
double or_normalised_residual(const or_grid *g, double *const cf[3], const double *b, const double *q) {
    int nc = g->ncell;
    double *Mq = calloc(nc, sizeof(double));
    double *ones = calloc(nc, sizeof(double));
    double *Mb = calloc(nc, sizeof(double));
    or_poisson_apply(g, cf, q, Mq);
    double qbar = 0.0;
    int m = 0;
    for (int c = 0; c < nc; ++c)
        if (!g->solid[c]) { qbar += q[c]; ++m; ones[c] = 1.0; }
    qbar /= (m > 0 ? m : 1);
    or_poisson_apply(g, cf, ones, Mb); /* M applied to the constant field 1 */
    double res = 0.0, nrm = 0.0;
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) continue;
        double Mqbar = qbar * Mb[c];
        res += fabs(b[c] - Mq[c]);
        nrm += fabs(Mq[c] - Mqbar) + fabs(b[c] - Mqbar);
    }
    free(Mq); free(ones); free(Mb);
    return res / (nrm + 1e-20);
}

/* ------------------------------------------------------------------------- */
/* PISO for one momentum equation (Section 2.2 with Eqs. NSE1d / NSEc).       */
/* The conservative ddt and convection terms are taken in their advective     */
/* equivalent (the conservative form minus v times the continuity equation): */
/*   rho_new (v - v_old)/dt + rho_new (phic . grad) v = -grad q               */
/*     + div(mu_new (grad v + grad v^T)) [+ sigma kappa grad alpha]           */
/* because in the split scheme alpha is carried by one flux (u_cr or u_vd)    */
/* while momentum is carried by u_vd + u_cr, so the discrete mass flux of the */
/* conservative form does not match the density change of the cell.          */
/* ------------------------------------------------------------------------- */
typedef struct {
    double E;       /* normalised initial residual of corrector 1 */
    int cg_iters;   /* total CG iterations */
    int cg_fail;
} piso_out;

/* face value of velocity component comp at face (a,s) of cell c: interior
 * average, wall 0, inlet vin, outlet zero-gradient */
static double vel_face_value(const or_grid *g, double *const v[3], const double *vin, int c, int a, int s, int comp) {
    int f, nb;
    int t = cell_face(g, c, a, s, &f, &nb);
    if (t == OR_F_INTERIOR) return 0.5 * (v[comp][c] + v[comp][nb]);
    if (t == OR_F_INLET) return vin[comp];
    if (t == OR_F_OUTLET) return v[comp][c];
    return 0.0;
}

/* HbyA = H / A for the current velocity iterate v: H holds the old-time term,
 * the neighbour part of the viscous Laplacian, the neighbour (inflow) part of
 * the upwind convection, the explicit linear-upwind correction (advective
 * form) and the explicit transpose viscous term div(mu grad v^T); the
 * outflow part of upwind convection sits in A (implicit). G receives the
 * Gauss gradients G[comp][dir] of v. */
static void momentum_HbyA(const or_grid *g, double *const v[3], double *const v_old[3],
                          double *const phic[3], const double *rho_n, const double *mu_n,
                          const double *rA, const double vin[3], double dt,
                          double *G[3][3], double *HbyA[3]) {
    int nc = g->ncell, D = g->dim;
    /* Gauss gradients of the current velocity: G[comp][dir] */
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) continue;
        for (int comp = 0; comp < D; ++comp)
            for (int dir = 0; dir < D; ++dir)
                G[comp][dir][c] = (vel_face_value(g, v, vin, c, dir, 1, comp) -
                                   vel_face_value(g, v, vin, c, dir, 0, comp)) / g->h[dir];
    }
    /* H and HbyA */
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) continue;
        for (int comp = 0; comp < D; ++comp) {
            double Hc = rho_n[c] * v_old[comp][c] / dt;
            double lap = 0.0, conv = 0.0, tr = 0.0, inflow = 0.0;
            for (int a = 0; a < D; ++a)
                for (int s = 0; s < 2; ++s) {
                    int f, nb;
                    int t = cell_face(g, c, a, s, &f, &nb);
                    double sg = s ? 1.0 : -1.0;
                    if (t == OR_F_INTERIOR) {
                        double muf = 0.5 * (mu_n[c] + mu_n[nb]);
                        lap += muf * g->S[a] / g->h[a] * v[comp][nb];
                        /* upwind (implicit part) and linear-upwind (explicit correction) face
                         * values for the convecting flux phic (oriented +a) */
                        int L = s ? c : nb, Hh = s ? nb : c;
                        double vf, vu;
                        if (phic[a][f] >= 0.0) { vu = v[comp][L]; vf = vu + 0.5 * g->h[a] * G[comp][a][L]; }
                        else { vu = v[comp][Hh]; vf = vu - 0.5 * g->h[a] * G[comp][a][Hh]; }
                        double fo = sg * phic[a][f];       /* outward flux of cell c */
                        if (fo < 0.0) inflow += -fo * v[comp][nb];
                        conv += fo * (vf - vu);
                        double dvdx = 0.5 * (G[a][comp][c] + G[a][comp][nb]);
                        tr += sg * muf * g->S[a] * dvdx;
                    } else if (t == OR_F_WALL) {
                        tr += sg * mu_n[c] * g->S[a] * G[a][comp][c];
                    } else if (t == OR_F_INLET) {
                        lap += mu_n[c] * g->S[a] / (0.5 * g->h[a]) * vin[comp];
                        double fo = sg * phic[a][f];
                        if (fo < 0.0) inflow += -fo * vin[comp];
                        else conv += fo * (vin[comp] - v[comp][c]);
                        tr += sg * mu_n[c] * g->S[a] * G[a][comp][c];
                    } else if (t == OR_F_OUTLET) {
                        tr += sg * mu_n[c] * g->S[a] * G[a][comp][c];
                    }
                }
            Hc += (lap + rho_n[c] * (inflow - conv) + tr) / g->V;
            HbyA[comp][c] = rA[c] * Hc;
        }
    }
}

static void piso(const or_grid *g, const or_params *P,
                 double *v[3], double *const v_old[3], double *q, double *phi[3], double *const phic[3],
                 const double *alpha_old, const double *alpha_new, const double *kappa, double sigma,
                 const double vin[3], double dt, piso_out *out) {
    int nc = g->ncell, D = g->dim;
    double *rho_n = calloc(nc, sizeof(double));
    double *mu_n = calloc(nc, sizeof(double)), *rA = calloc(nc, sizeof(double));
    double *b = calloc(nc, sizeof(double));
    double *HbyA[3] = {0}, *G[3][3] = {{0}}, *cf[3] = {0}, *fst[3] = {0}, *phis[3] = {0};
    for (int a = 0; a < 3; ++a) {
        HbyA[a] = calloc(nc, sizeof(double));
        for (int b2 = 0; b2 < 3; ++b2) G[a][b2] = calloc(nc, sizeof(double));
        cf[a] = calloc(g->nface[a], sizeof(double));
        fst[a] = calloc(g->nface[a], sizeof(double));
        phis[a] = calloc(g->nface[a], sizeof(double));
    }
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) continue;
        rho_n[c] = mix_rho(P, alpha_new[c]);
        mu_n[c] = mix_mu(P, alpha_new[c]);
    }
    /* diagonal A = rho_new/dt + (1/V) sum mu_f S/delta over interior, wall and inlet faces
     * + (rho_new/V) sum of the inflow fluxes (implicit upwind part of convection) */
    for (int c = 0; c < nc; ++c) {
        if (g->solid[c]) continue;
        double acc = 0.0, cin = 0.0;
        for (int a = 0; a < D; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                int t = cell_face(g, c, a, s, &f, &nb);
                if (t == OR_F_INTERIOR) acc += 0.5 * (mu_n[c] + mu_n[nb]) * g->S[a] / g->h[a];
                else if (t == OR_F_WALL || t == OR_F_INLET) acc += mu_n[c] * g->S[a] / (0.5 * g->h[a]);
                if (t == OR_F_INTERIOR || t == OR_F_INLET) {
                    double fo = (s ? 1.0 : -1.0) * phic[a][f];
                    if (fo < 0.0) cin += -fo;
                }
            }
        rA[c] = 1.0 / (rho_n[c] / dt + (acc + rho_n[c] * cin) / g->V);
    }
    /* face coefficients of the pressure operator, CSF face forces */
    for (int a = 0; a < D; ++a) {
        FOR_FACES(g, a, fijk, f) {
            int L, H;
            int t = face_cells(g, a, fijk, &L, &H);
            if (t == OR_F_INTERIOR) {
                cf[a][f] = 0.5 * (rA[L] + rA[H]) * g->S[a] / g->h[a];
                if (kappa)
                    fst[a][f] = sigma * 0.5 * (kappa[L] + kappa[H]) * (alpha_new[H] - alpha_new[L]) / g->h[a];
            } else if (t == OR_F_OUTLET) {
                cf[a][f] = rA[L] * g->S[a] / (0.5 * g->h[a]);
            }
        }
    }
    out->cg_iters = 0;
    out->cg_fail = 0;
    out->E = 0.0;
    for (int corr = 0; corr < P->n_piso; ++corr) {
        momentum_HbyA(g, v, v_old, phic, rho_n, mu_n, rA, vin, dt, G, HbyA);
        /* predicted fluxes phi* and right-hand side b = -div(phi*) */
        for (int a = 0; a < D; ++a) {
            FOR_FACES(g, a, fijk, f) {
                int L, H;
                int t = face_cells(g, a, fijk, &L, &H);
                double ps = 0.0;
                if (t == OR_F_INTERIOR)
                    ps = 0.5 * (HbyA[a][L] + HbyA[a][H]) * g->S[a] + 0.5 * (rA[L] + rA[H]) * fst[a][f] * g->S[a];
                else if (t == OR_F_INLET) ps = vin[a] * g->S[a];
                else if (t == OR_F_OUTLET) ps = HbyA[a][L] * g->S[a];
                phis[a][f] = ps;
            }
        }
        for (int c = 0; c < nc; ++c) {
            if (g->solid[c]) { b[c] = 0.0; continue; }
            double div = 0.0;
            for (int a = 0; a < D; ++a)
                for (int s = 0; s < 2; ++s) {
                    int f, nb;
                    cell_face(g, c, a, s, &f, &nb);
                    div += s ? phis[a][f] : -phis[a][f];
                }
            b[c] = -div;
        }
        if (corr == 0) out->E = or_normalised_residual(g, cf, b, q);
        /* the pressure equation is solved exactly (banded Cholesky) where the
         * band is narrow, else by Jacobi-PCG to cg_rtol */
        int it = 0;
        if (or_poisson_banded(g, cf, b, q, OR_BANDED_MAX_WORK) != 0) {
            it = or_poisson_cg(g, cf, b, q, P->cg_rtol, P->cg_maxit);
            if (it < 0) { out->cg_fail = 1; it = -it; }
        }
        out->cg_iters += it;
        /* flux correction phi = phi* - c_f (q_H - q_L) */
        for (int a = 0; a < D; ++a) {
            FOR_FACES(g, a, fijk, f) {
                int L, H;
                int t = face_cells(g, a, fijk, &L, &H);
                if (t == OR_F_INTERIOR) phi[a][f] = phis[a][f] - cf[a][f] * (q[H] - q[L]);
                else if (t == OR_F_OUTLET) phi[a][f] = phis[a][f] - cf[a][f] * (0.0 - q[L]);
                else phi[a][f] = phis[a][f];
            }
        }
        /* velocity correction v = HbyA + rA * reconstruct(face accelerations) */
        for (int c = 0; c < nc; ++c) {
            if (g->solid[c]) continue;
            for (int a = 0; a < D; ++a) {
                double gs = 0.0;
                for (int s = 0; s < 2; ++s) {
                    int f, nb;
                    int t = cell_face(g, c, a, s, &f, &nb);
                    if (t == OR_F_INTERIOR) {
                        int L = s ? c : nb, Hh = s ? nb : c;
                        gs += fst[a][f] - (q[Hh] - q[L]) / g->h[a];
                    } else if (t == OR_F_OUTLET) {
                        gs += -(0.0 - q[c]) / (0.5 * g->h[a]);
                    }
                }
                v[a][c] = HbyA[a][c] + rA[c] * 0.5 * gs;
            }
        }
    }
    free(rho_n); free(mu_n); free(rA); free(b);
    for (int a = 0; a < 3; ++a) {
        free(HbyA[a]);
        for (int b2 = 0; b2 < 3; ++b2) free(G[a][b2]);
        free(cf[a]); free(fst[a]); free(phis[a]);
    }
}

/* ------------------------------------------------------------------------- */
/* state: create / drag / relax / standard / fields                          */
/* ------------------------------------------------------------------------- */
or_state *or_create(const or_params *P, const uint8_t *solid, const double *alpha0) {
    or_state *S = calloc(1, sizeof(or_state));
    S->P = *P;
    int ncell = P->nx * P->ny * (P->dim == 3 ? P->nz : 1);
    S->solid = malloc(ncell);
    memcpy(S->solid, solid, ncell);
    grid_init(&S->g, P, S->solid);
    or_grid *g = &S->g;
    S->alpha = calloc(ncell, sizeof(double));
    S->kappa = calloc(ncell, sizeof(double));
    S->alpha_s = calloc(ncell, sizeof(double));
    S->p_vd = calloc(ncell, sizeof(double));
    S->p_cr = calloc(ncell, sizeof(double));
    for (int a = 0; a < 3; ++a) {
        S->nf[a] = calloc(g->nface[a], sizeof(double));
        S->phi_vd[a] = calloc(g->nface[a], sizeof(double));
        S->phi_cr[a] = calloc(g->nface[a], sizeof(double));
        S->u_vd[a] = calloc(ncell, sizeof(double));
        S->u_cr[a] = calloc(ncell, sizeof(double));
        S->u_cr_sum[a] = calloc(ncell, sizeof(double));
    }
    for (int c = 0; c < ncell; ++c) S->alpha[c] = solid[c] ? 0.0 : alpha0[c];
    or_interface(g, S->alpha, P->n_smooth, P->theta_deg, S->alpha_s, S->nf, S->kappa);
    S->last_N = 1;
    return S;
}

void or_destroy(or_state *S) {
    if (!S) return;
    free(S->solid); free(S->alpha); free(S->kappa); free(S->alpha_s); free(S->p_vd); free(S->p_cr);
    for (int a = 0; a < 3; ++a) {
        free(S->nf[a]); free(S->phi_vd[a]); free(S->phi_cr[a]);
        free(S->u_vd[a]); free(S->u_cr[a]); free(S->u_cr_sum[a]);
    }
    free(S);
}

static double **dup_fields(const or_grid *g, double *const src[3], int faces) {
    double **d = calloc(3, sizeof(double *));
    for (int a = 0; a < 3; ++a) {
        size_t n = faces ? g->nface[a] : g->ncell;
        d[a] = malloc(n * sizeof(double));
        memcpy(d[a], src[a], n * sizeof(double));
    }
    return d;
}

static void free_fields(double **d) {
    for (int a = 0; a < 3; ++a) free(d[a]);
    free(d);
}

/* Section 3.1: viscous-drag step (Eqs. VOFd, NSE1d, md). alpha^n -> alpha* with
 * u_vd^n; momentum for u_vd with convecting flux phi_vd^n + phi_cr^n, no
 * surface tension, inlet velocity U. */
int or_drag_step(or_state *S, double dt) {
    or_grid *g = &S->g;
    const or_params *P = &S->P;
    int nc = g->ncell;
    double *alpha_new = calloc(nc, sizeof(double));
    or_transport(g, S->alpha, S->phi_vd, S->nf, dt, P->c_alpha, P->alpha_inlet, alpha_new);
    double **phic = calloc(3, sizeof(double *));
    for (int a = 0; a < 3; ++a) {
        phic[a] = malloc(g->nface[a] * sizeof(double));
        for (int f = 0; f < g->nface[a]; ++f) phic[a][f] = S->phi_vd[a][f] + S->phi_cr[a][f];
    }
    double **vold = dup_fields(g, S->u_vd, 0);
    double vin[3] = {P->U_inlet, 0.0, 0.0};
    piso_out po;
    piso(g, P, S->u_vd, vold, S->p_vd, S->phi_vd, phic, S->alpha, alpha_new, NULL, 0.0, vin, dt, &po);
    memcpy(S->alpha, alpha_new, nc * sizeof(double));
    or_interface(g, S->alpha, P->n_smooth, P->theta_deg, S->alpha_s, S->nf, S->kappa);
    S->cg_iters_last = po.cg_iters;
    S->cg_iters_total += po.cg_iters;
    S->cg_fail |= po.cg_fail;
    free_fields(phic); free_fields(vold); free(alpha_new);
    return po.cg_fail ? -3 : 0;
}

/* Interface area A = sum over fluid cells of |grad alpha| V, with the Gauss
 * gradient of alpha (face values: the mean of the two cells on interior faces,
 * the cell's own value on boundary faces). */
double or_interface_area(const or_grid *g, const double *alpha) {
    double A = 0.0;
    for (int c = 0; c < g->ncell; ++c) {
        if (g->solid[c]) continue;
        double m2 = 0.0;
        for (int b = 0; b < g->dim; ++b) {
            double gb = gauss_grad_scalar(g, alpha, c, b);
            m2 += gb * gb;
        }
        A += sqrt(m2) * g->V;
    }
    return A;
}

/* Mechanical energy of the relaxation: interfacial energy sigma A plus the
 * kinetic energy of the capillary velocity, sum over fluid cells of
 * rho(alpha) |u|^2 V / 2 (Section 2.1 mixture density). Section 6 suggests
 * identifying capillary equilibrium by an energy balance; the relaxation's
 * energy test is the relative change of this energy over a sub-step. */
double or_relax_energy(const or_grid *g, const or_params *P, const double *alpha, double *const *u) {
    double K = 0.0;
    for (int c = 0; c < g->ncell; ++c) {
        if (g->solid[c]) continue;
        double u2 = 0.0;
        for (int a = 0; a < g->dim; ++a) u2 += u[a][c] * u[a][c];
        K += 0.5 * mix_rho(P, alpha[c]) * u2 * g->V;
    }
    return P->sigma * or_interface_area(g, alpha) + K;
}

/* Section 3.2: capillary-relaxation sub-steps (Eqs. VOFc, NSEc, mc) with the
 * early exit on E_k (or on the max velocity change), then the reconstruction
 * of u^{n+1} = u_vd + (1/N) sum_k u_cr^{n,k}. E_hist (may be NULL) receives
 * the test value of each sub-step. */
int or_relax(or_state *S, double dt_cr, int N, int *kf_out, double *E_hist) {
    or_grid *g = &S->g;
    const or_params *P = &S->P;
    int nc = g->ncell, D = g->dim;
    double *alpha_new = calloc(nc, sizeof(double));
    double vin[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) memset(S->u_cr_sum[a], 0, nc * sizeof(double));
    int kf = 0, fail = 0;
    double energy_old = (P->conv_mode == OR_CONV_AREA) ? or_relax_energy(g, P, S->alpha, S->u_cr) : 0.0;
    for (int k = 0; k < N; ++k) {
        or_transport(g, S->alpha, S->phi_cr, S->nf, dt_cr, P->c_alpha, P->alpha_inlet, alpha_new);
        or_interface(g, alpha_new, P->n_smooth, P->theta_deg, S->alpha_s, S->nf, S->kappa);
        double **phic = calloc(3, sizeof(double *));
        for (int a = 0; a < 3; ++a) {
            phic[a] = malloc(g->nface[a] * sizeof(double));
            for (int f = 0; f < g->nface[a]; ++f) phic[a][f] = S->phi_vd[a][f] + S->phi_cr[a][f];
        }
        double **vold = dup_fields(g, S->u_cr, 0);
        piso_out po;
        piso(g, P, S->u_cr, vold, S->p_cr, S->phi_cr, phic, S->alpha, alpha_new, S->kappa, P->sigma,
             vin, dt_cr, &po);
        memcpy(S->alpha, alpha_new, nc * sizeof(double));
        double dU = 0.0;
        for (int a = 0; a < D; ++a)
            for (int c = 0; c < nc; ++c) {
                if (g->solid[c]) continue;
                S->u_cr_sum[a][c] += S->u_cr[a][c];
                double d = fabs(S->u_cr[a][c] - vold[a][c]);
                if (d > dU) dU = d;
            }
        dU /= P->U_inlet;
        S->cg_iters_last = po.cg_iters;
        S->cg_iters_total += po.cg_iters;
        fail |= po.cg_fail;
        free_fields(phic); free_fields(vold);
        kf = k + 1;
        double test = (P->conv_mode == OR_CONV_DU_MAX) ? dU : po.E;
        if (P->conv_mode == OR_CONV_AREA) {   /* relative change of the energy (Section 6) */
            double energy = or_relax_energy(g, P, S->alpha, S->u_cr);
            test = fabs(energy - energy_old) / (energy_old > 0.0 ? energy_old : 1.0);
            energy_old = energy;
        }
        if (E_hist) E_hist[k] = test;
        S->last_E = po.E;
        S->last_dU = dU;
        if (test < P->conv_tol) break;
    }
    S->last_kf = kf;
    S->last_N = N;
    S->cg_fail |= fail;
    if (kf_out) *kf_out = kf;
    free(alpha_new);
    return fail ? -3 : 0;
}

/* Standard time-stepping (Section 2.2): one explicit alpha step with u^n, then
 * PISO with surface tension and the inlet velocity. The drag-step fields hold
 * u, p, phi in this mode; the relaxation fields stay zero. */
int or_standard_step(or_state *S, double dt) {
    or_grid *g = &S->g;
    const or_params *P = &S->P;
    int nc = g->ncell;
    double *alpha_new = calloc(nc, sizeof(double));
    or_transport(g, S->alpha, S->phi_vd, S->nf, dt, P->c_alpha, P->alpha_inlet, alpha_new);
    or_interface(g, alpha_new, P->n_smooth, P->theta_deg, S->alpha_s, S->nf, S->kappa);
    double **phic = dup_fields(g, S->phi_vd, 1);
    double **vold = dup_fields(g, S->u_vd, 0);
    double vin[3] = {P->U_inlet, 0.0, 0.0};
    piso_out po;
    piso(g, P, S->u_vd, vold, S->p_vd, S->phi_vd, phic, S->alpha, alpha_new, S->kappa, P->sigma,
         vin, dt, &po);
    memcpy(S->alpha, alpha_new, nc * sizeof(double));
    for (int a = 0; a < 3; ++a) memset(S->u_cr_sum[a], 0, nc * sizeof(double));
    S->last_E = po.E;
    S->last_N = 1;
    S->cg_iters_last = po.cg_iters;
    S->cg_iters_total += po.cg_iters;
    S->cg_fail |= po.cg_fail;
    free_fields(phic); free_fields(vold); free(alpha_new);
    return po.cg_fail ? -3 : 0;
}

/* Field read-out. which: 0 alpha, 1 p = p_vd + p_cr, 2..4 u (reported,
 * u_vd + sum u_cr / N), 5..7 u_vd, 8..10 u_cr, 11 p_vd, 12 p_cr, 13 kappa,
 * 14..16 phi_vd (faces), 17..19 phi_cr (faces), 20..22 nf (faces). */
int or_field(const or_state *S, int which, double *out) {
    const or_grid *g = &S->g;
    int nc = g->ncell;
    if (which == 0) { memcpy(out, S->alpha, nc * sizeof(double)); return nc; }
    if (which == 1) { for (int c = 0; c < nc; ++c) out[c] = S->p_vd[c] + S->p_cr[c]; return nc; }
    if (which >= 2 && which <= 4) {
        int a = which - 2;
        for (int c = 0; c < nc; ++c) out[c] = S->u_vd[a][c] + S->u_cr_sum[a][c] / S->last_N;
        return nc;
    }
    if (which >= 5 && which <= 7) { memcpy(out, S->u_vd[which - 5], nc * sizeof(double)); return nc; }
    if (which >= 8 && which <= 10) { memcpy(out, S->u_cr[which - 8], nc * sizeof(double)); return nc; }
    if (which == 11) { memcpy(out, S->p_vd, nc * sizeof(double)); return nc; }
    if (which == 12) { memcpy(out, S->p_cr, nc * sizeof(double)); return nc; }
    if (which == 13) { memcpy(out, S->kappa, nc * sizeof(double)); return nc; }
    if (which >= 14 && which <= 16) { int a = which - 14; memcpy(out, S->phi_vd[a], g->nface[a] * sizeof(double)); return g->nface[a]; }
    if (which >= 17 && which <= 19) { int a = which - 17; memcpy(out, S->phi_cr[a], g->nface[a] * sizeof(double)); return g->nface[a]; }
    if (which >= 20 && which <= 22) { int a = which - 20; memcpy(out, S->nf[a], g->nface[a] * sizeof(double)); return g->nface[a]; }
    return -1;
}

/* Overwrite state fields (for stage tests and checkpoint-style restarts);
 * same numbering as or_field; 1 sets p_vd, 2..4 are not accepted. */
int or_set_field(or_state *S, int which, const double *in) {
    or_grid *g = &S->g;
    int nc = g->ncell;
    if (which == 0) {
        memcpy(S->alpha, in, nc * sizeof(double));
        or_interface(g, S->alpha, S->P.n_smooth, S->P.theta_deg, S->alpha_s, S->nf, S->kappa);
        return nc;
    }
    if (which >= 5 && which <= 7) { memcpy(S->u_vd[which - 5], in, nc * sizeof(double)); return nc; }
    if (which >= 8 && which <= 10) { memcpy(S->u_cr[which - 8], in, nc * sizeof(double)); return nc; }
    if (which == 11 || which == 1) { memcpy(S->p_vd, in, nc * sizeof(double)); return nc; }
    if (which == 12) { memcpy(S->p_cr, in, nc * sizeof(double)); return nc; }
    if (which >= 14 && which <= 16) { int a = which - 14; memcpy(S->phi_vd[a], in, g->nface[a] * sizeof(double)); return g->nface[a]; }
    if (which >= 17 && which <= 19) { int a = which - 17; memcpy(S->phi_cr[a], in, g->nface[a] * sizeof(double)); return g->nface[a]; }
    return -1;
}

void or_stats(const or_state *S, double *out) {
    double vol = 0.0;
    for (int c = 0; c < S->g.ncell; ++c)
        if (!S->g.solid[c]) vol += S->alpha[c] * S->g.V;
    out[0] = S->last_kf;
    out[1] = S->last_E;
    out[2] = S->last_dU;
    out[3] = (double)S->cg_iters_total;
    out[4] = S->cg_iters_last;
    out[5] = vol;
    out[6] = S->cg_fail;
}

/* ------------------------------------------------------------------------- */
/* stage entry points on plain arrays (for pins)                              */
/* ------------------------------------------------------------------------- */
void or_stage_transport(const or_params *P, const uint8_t *solid, const double *alpha,
                        double *phix, double *phiy, double *phiz,
                        double *nfx, double *nfy, double *nfz, double dt, double *alpha_new) {
    or_grid g;
    grid_init(&g, P, solid);
    double *phi[3] = {phix, phiy, phiz};
    double *nf[3] = {nfx, nfy, nfz};
    or_transport(&g, alpha, phi, nf, dt, P->c_alpha, P->alpha_inlet, alpha_new);
}

void or_stage_interface(const or_params *P, const uint8_t *solid, const double *alpha,
                        double *alpha_s, double *nfx, double *nfy, double *nfz, double *kappa) {
    or_grid g;
    grid_init(&g, P, solid);
    double *nf[3] = {nfx, nfy, nfz};
    or_interface(&g, alpha, P->n_smooth, P->theta_deg, alpha_s, nf, kappa);
}

double or_stage_interface_area(const or_params *P, const uint8_t *solid, const double *alpha) {
    or_grid g;
    grid_init(&g, P, solid);
    return or_interface_area(&g, alpha);
}

double or_stage_relax_energy(const or_params *P, const uint8_t *solid, const double *alpha, double *ux,
                             double *uy, double *uz) {
    or_grid g;
    grid_init(&g, P, solid);
    double *u[3] = {ux, uy, uz};
    return or_relax_energy(&g, P, alpha, u);
}

void or_stage_poisson_apply(const or_params *P, const uint8_t *solid, double *cx, double *cy, double *cz,
                            const double *q, double *y) {
    or_grid g;
    grid_init(&g, P, solid);
    double *cf[3] = {cx, cy, cz};
    or_poisson_apply(&g, cf, q, y);
}

int or_stage_poisson_cg(const or_params *P, const uint8_t *solid, double *cx, double *cy, double *cz,
                        const double *b, double *q, double rtol, int maxit) {
    or_grid g;
    grid_init(&g, P, solid);
    double *cf[3] = {cx, cy, cz};
    return or_poisson_cg(&g, cf, b, q, rtol, maxit);
}

int or_stage_poisson_dense(const or_params *P, const uint8_t *solid, double *cx, double *cy, double *cz,
                           const double *b, double *q) {
    or_grid g;
    grid_init(&g, P, solid);
    double *cf[3] = {cx, cy, cz};
    return or_poisson_dense(&g, cf, b, q);
}

double or_stage_normalised_residual(const or_params *P, const uint8_t *solid, double *cx, double *cy,
                                    double *cz, const double *b, const double *q) {
    or_grid g;
    grid_init(&g, P, solid);
    double *cf[3] = {cx, cy, cz};
    return or_normalised_residual(&g, cf, b, q);
}

/* One PISO solve on plain arrays: v (3 cell arrays, in/out), q (in/out), phi
 * (3 face arrays, out), phic (convecting flux), kappa may be NULL. out3 gets
 * {E, cg_iters, cg_fail}. */
void or_stage_piso(const or_params *P, const uint8_t *solid,
                   double *vx, double *vy, double *vz, double *vox, double *voy, double *voz,
                   double *q, double *phx, double *phy, double *phz,
                   double *pcx, double *pcy, double *pcz,
                   const double *alpha_old, const double *alpha_new, const double *kappa,
                   double vin_x, double dt, double *out3) {
    or_grid g;
    grid_init(&g, P, solid);
    double *v[3] = {vx, vy, vz}, *vo[3] = {vox, voy, voz}, *ph[3] = {phx, phy, phz}, *pc[3] = {pcx, pcy, pcz};
    double vin[3] = {vin_x, 0.0, 0.0};
    piso_out po;
    piso(&g, P, v, vo, q, ph, pc, alpha_old, alpha_new, kappa, P->sigma, vin, dt, &po);
    out3[0] = po.E;
    out3[1] = po.cg_iters;
    out3[2] = po.cg_fail;
}

/* One evaluation of HbyA and rA for given fields (for pins of the momentum
 * terms). hbya: 3 cell arrays out; rA_out: cell array out. */
void or_stage_momentum(const or_params *P, const uint8_t *solid,
                       double *vx, double *vy, double *vz, double *vox, double *voy, double *voz,
                       double *pcx, double *pcy, double *pcz, const double *alpha_new,
                       double vin_x, double dt, double *hx, double *hy, double *hz, double *rA_out) {
    or_grid g;
    grid_init(&g, P, solid);
    int nc = g.ncell, D = g.dim;
    double *v[3] = {vx, vy, vz}, *vo[3] = {vox, voy, voz}, *pc[3] = {pcx, pcy, pcz};
    double *HbyA[3] = {hx, hy, hz};
    double vin[3] = {vin_x, 0.0, 0.0};
    double *rho_n = calloc(nc, sizeof(double)), *mu_n = calloc(nc, sizeof(double));
    double *G[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] = calloc(nc, sizeof(double));
    for (int c = 0; c < nc; ++c) {
        if (g.solid[c]) continue;
        rho_n[c] = mix_rho(P, alpha_new[c]);
        mu_n[c] = mix_mu(P, alpha_new[c]);
    }
    for (int c = 0; c < nc; ++c) {
        if (g.solid[c]) continue;
        double acc = 0.0, cin = 0.0;
        for (int a = 0; a < D; ++a)
            for (int s = 0; s < 2; ++s) {
                int f, nb;
                int t = cell_face(&g, c, a, s, &f, &nb);
                if (t == OR_F_INTERIOR) acc += 0.5 * (mu_n[c] + mu_n[nb]) * g.S[a] / g.h[a];
                else if (t == OR_F_WALL || t == OR_F_INLET) acc += mu_n[c] * g.S[a] / (0.5 * g.h[a]);
                if (t == OR_F_INTERIOR || t == OR_F_INLET) {
                    double fo = (s ? 1.0 : -1.0) * pc[a][f];
                    if (fo < 0.0) cin += -fo;
                }
            }
        rA_out[c] = 1.0 / (rho_n[c] / dt + (acc + rho_n[c] * cin) / g.V);
    }
    momentum_HbyA(&g, v, vo, pc, rho_n, mu_n, rA_out, vin, dt, G, HbyA);
    free(rho_n); free(mu_n);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) free(G[a][b]);
}

int or_stage_poisson_banded(const or_params *P, const uint8_t *solid, double *cx, double *cy, double *cz,
                            const double *b, double *q) {
    or_grid g;
    grid_init(&g, P, solid);
    double *cf[3] = {cx, cy, cz};
    return or_poisson_banded(&g, cf, b, q, 1e18);
}
