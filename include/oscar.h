/*
 * oscar.h - C ABI of the GB300 (sm_103a) implementation of OSCAR, Operator
 * Splitting with Capillary Relaxation (Maes & Menke, arXiv 2105.10576), on a
 * uniform voxel grid with a solid mask.
 *
 * One handle holds one simulation instance: every field, face flux and
 * multigrid level of it lives in device memory owned by the library. All
 * arguments are plain host values or host pointers unless a name ends in
 * "_device". Calls on one handle are ordered on the CUDA stream given at
 * creation; calls that return host data wait for that stream with a bounded
 * wait (OSCAR_E_TIMEOUT after 600 s). No call aborts the process or traps the
 * device. Calls on one handle are not thread-safe; distinct handles are
 * independent.
 *
 * Conventions (shared by every entry point):
 *   - cells are indexed c = i + nx*(j + ny*k), x fastest; 2D grids have nz = 1;
 *   - solid[c] = 1 marks a solid cell; fluid/solid faces and the y/z domain
 *     boundaries are walls; x-min is the inlet, x-max the outlet (Section 3:
 *     inlet with constant injected velocity, free outlet, no-slip walls);
 *   - face arrays of direction a hold the faces on the low side of every cell
 *     plus one extra layer: (nx+1)*ny*nz x-faces, nx*(ny+1)*nz y-faces,
 *     nx*ny*(nz+1) z-faces, fluxes oriented along +a;
 *   - alpha = 1 is phase 1 (rho1, mu1); theta_deg is measured through phase 1.
 *
 * Return codes: 0 on success, a negative OSCAR_E_* value otherwise. After
 * OSCAR_E_CUDA the handle may only be destroyed.
 */
#ifndef OSCAR_H
#define OSCAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OSCAR_OK 0
#define OSCAR_E_INVALID_ARG (-1)
#define OSCAR_E_OOM (-2)
#define OSCAR_E_NOT_CONVERGED (-3)
#define OSCAR_E_NAN (-4)
#define OSCAR_E_TIMEOUT (-5)
#define OSCAR_E_CUDA (-6)

#define OSCAR_FP64 0  /* every field and solve in FP64 */
#define OSCAR_MIXED 1 /* FP32 fields, stencils and V-cycles; FP64 CG vectors, dots, norms, sums */

#define OSCAR_CONV_PRES_RESID 0 /* E_k: normalised initial residual of PISO corrector 1 (Section 3.2) */
#define OSCAR_CONV_DU_MAX 1     /* max |u_cr^{k+1} - u_cr^k| / U_inlet */
#define OSCAR_CONV_AREA 2       /* |E^k - E^{k-1}| / E^{k-1}, E = sigma A + sum rho |u_cr|^2 V / 2 with
                                   A = sum over fluid cells of |grad alpha| V: the relaxation's energy
                                   stationary (an energy-balance test of capillary equilibrium, a
                                   variant suggested in Section 6, not the published method) */

/* Field selectors for oscar_fields / oscar_set_field. */
#define OSCAR_FIELD_ALPHA 0
#define OSCAR_FIELD_P 1      /* p = p_vd + p_cr (Section 3.2 reconstruction) */
#define OSCAR_FIELD_U 2      /* 2,3,4: u = u_vd + (1/N) sum_k u_cr^{n,k} */
#define OSCAR_FIELD_U_VD 5   /* 5,6,7 */
#define OSCAR_FIELD_U_CR 8   /* 8,9,10 */
#define OSCAR_FIELD_P_VD 11
#define OSCAR_FIELD_P_CR 12
#define OSCAR_FIELD_KAPPA 13
#define OSCAR_FIELD_PHI_VD 14 /* 14,15,16 (face arrays) */
#define OSCAR_FIELD_PHI_CR 17 /* 17,18,19 (face arrays) */
#define OSCAR_FIELD_NF 20     /* 20,21,22 face-normal component of the interface normal */

/* Problem statement and numerical parameters (Section 3, problem statement;
 * Sections 2.1-2.2 for the fluid model). Plain host struct, copied at
 * creation. */
typedef struct {
    int dim;               /* 2 or 3 */
    int nx, ny, nz;        /* cells per direction (nz = 1 in 2D) */
    double hx, hy, hz;     /* cell size [m] */
    double rho1, rho2;     /* densities [kg/m^3] of phase 1 (alpha = 1) and phase 2 */
    double mu1, mu2;       /* viscosities [Pa s] */
    double sigma;          /* interfacial tension [N/m] */
    double theta_deg;      /* static contact angle through phase 1 [deg] */
    double U_inlet;        /* injected velocity at x-min [m/s] */
    double alpha_inlet;    /* alpha of the injected fluid */
    int n_piso;            /* PISO correctors (3 in the paper, Section 2.2) */
    int n_smooth;          /* smoothing passes of alpha before the normal (2) */
    double c_alpha;        /* interface-compression coefficient (1) */
    int conv_mode;         /* OSCAR_CONV_* */
    double conv_tol;       /* relaxation tolerance (1e-4 for E_k in the paper) */
    double cg_rtol;        /* pressure solve: stop at ||r||_2 <= cg_rtol ||b||_2 */
    int cg_maxit;          /* pressure solve iteration cap */
    int precision;         /* OSCAR_FP64 or OSCAR_MIXED */
} oscar_params;

typedef struct {
    int k_f;                  /* sub-steps run in the last relaxation (Section 3.2) */
    int N;                    /* sub-steps allowed in the last relaxation */
    double E_last;            /* E_k of the last sub-step */
    double dU_last;           /* max |u_cr^{k+1} - u_cr^k| / U_inlet of the last sub-step */
    long long cg_iters_total; /* PCG iterations since creation */
    int cg_iters_last;        /* PCG iterations of the last step or sub-step */
    int mg_levels;            /* multigrid levels of the pressure preconditioner */
    double phase_volume;      /* sum over fluid cells of alpha V (FP64) */
    long long n_fluid;        /* fluid cells */
    long long cell_updates;   /* fluid cells x (drag + relaxation + standard steps) since creation */
    size_t device_bytes;      /* device memory held by the handle */
    long long kernel_launches; /* CUDA kernels launched by this handle since creation */
    int mg_first_cta_level;   /* first multigrid level held in one CTA's shared memory */
    int mg_cta_global_level;  /* level worked by that CTA with coefficients in global memory, -1 when none */
} oscar_stats_t;

typedef struct oscar_instance *oscar_handle;

/* Time-step control (Section 2.2, CFL and Brackbill limits; Section 3.2, N).
 * out[0] = dt_CFL = hx / u; out[1] = dt_B = sqrt(rho_bar h_min^3 / (2 pi sigma)),
 * rho_bar = (rho1 + rho2)/2, h_min the smallest spacing; out[2] = dt_vd = c_cfl dt_CFL;
 * out[3] = N, the smallest integer with dt_vd / N < dt_B.
 * u is the flow velocity of the CFL condition, fixed before the run from the
 * geometry: the injected flux U_inlet A(inlet) crosses every x cross-section,
 * so u = U_inlet A(inlet) / min_x A(x), A(x) = fluid cells of the column
 * i = const (the mean speed through the narrowest section; U_inlet in a
 * straight channel). solid: host uint8[ncell] (1 = solid), or NULL for a
 * grid without solid cells (u = U_inlet). Returns OSCAR_E_INVALID_ARG for
 * U_inlet, sigma or c_cfl not positive, or when the inlet column has fluid
 * but some column has none (no path to the outlet). Host arithmetic only. */
int oscar_timesteps(const oscar_params *p, const uint8_t *solid, double c_cfl, double out[4]);

/* Create an instance. solid: host uint8[ncell]; alpha0: host double[ncell]
 * (values in solid cells ignored). stream: a cudaStream_t, or NULL for a
 * stream the library creates and owns (the step graphs cannot be captured on
 * the legacy default stream). Velocities, pressures and fluxes start at zero
 * (fluid at rest). Allocates all device memory of the instance. The
 * environment variable OSCAR_EAGER=1 selects host-driven loops instead of
 * graphs (same kernels, one host read-back per loop trip; for per-kernel
 * profiling). */
int oscar_create(const oscar_params *p, const uint8_t *solid, const double *alpha0, void *stream,
                 oscar_handle *out);

/* Viscous-drag step (Section 3.1, Eqs. VOFd, NSE1d, md): alpha^n -> alpha*
 * with u_vd^n; momentum for u_vd with convecting velocity u_vd^n + u_cr^n,
 * no surface tension, inlet velocity U_inlet, outlet p_vd = 0; PISO. */
int oscar_drag_step(oscar_handle h, double dt_vd);

/* Capillary relaxation (Section 3.2, Eqs. VOFc, NSEc, mc): up to N sub-steps of
 * dt_cr, each an explicit alpha step with u_cr, the CSF force of the new alpha,
 * and PISO for u_cr (zero at the inlet) with convecting velocity u_vd + u_cr;
 * stops after sub-step k_f when the test value (E_k or max |du_cr|/U) is
 * below conv_tol, or at k_f = N. Then u = u_vd + (1/N) sum_{k<=k_f} u_cr^{n,k}.
 * k_f_out and test_out (may be NULL) receive k_f and the last test value. */
int oscar_relax(oscar_handle h, double dt_cr, int N, int *k_f_out, double *test_out);

/* Standard time-stepping (Section 2.2): one explicit alpha step with u^n, then
 * PISO with surface tension and the inlet velocity. In this mode the drag
 * fields (u_vd, p_vd, phi_vd) hold u, p, phi and the relaxation fields stay 0. */
int oscar_standard_step(oscar_handle h, double dt);

/* Device memory (bytes) that oscar_create would allocate for these parameters,
 * from the same layout computation and without allocating anything (for
 * admission control by memory footprint). Errors as oscar_create's parameter
 * validation. Not part of the paper's method. */
int oscar_footprint(const oscar_params *p, size_t *bytes_out);

/* Asynchronous forms of the three steps: each validates its arguments, launches
 * the step on the handle's stream (one CUDA graph launch, plus the copies of its
 * loop counters back to pinned host memory) and returns without waiting, so that
 * the steps of many handles, each on its own stream, run at the same time on the
 * GPU. A handle with a launched step accepts only oscar_wait and oscar_destroy
 * (every other call returns OSCAR_E_INVALID_ARG) until oscar_wait has collected
 * it. Arguments and errors as for the synchronous calls; launch failures are
 * returned here, the step's own status by oscar_wait. These belong to the
 * serving/batching layer, not to the paper's method. */
int oscar_drag_step_async(oscar_handle h, double dt_vd);
int oscar_relax_async(oscar_handle h, double dt_cr, int N);
int oscar_standard_step_async(oscar_handle h, double dt);

/* Non-blocking check of the step launched by an *_async call: 1 when it has
 * finished (oscar_wait then returns at once), 0 while it runs, OSCAR_E_INVALID_ARG
 * when no step is pending, OSCAR_E_CUDA on a stream error. */
int oscar_query(oscar_handle h);

/* Wait (bounded, OSCAR_E_TIMEOUT after 600 s) for the step launched by an
 * *_async call and return its status as the synchronous call would. k_f_out
 * (may be NULL) receives k_f for a relaxation, 1 otherwise; test_out (may be
 * NULL) the last test value of a relaxation, else the step's E. Returns
 * OSCAR_E_INVALID_ARG when no step is pending. */
int oscar_wait(oscar_handle h, int *k_f_out, double *test_out);

/* Copy one field to host memory (double). n must equal the field's length
 * (ncell, or the face count of its direction). Waits for the stream. */
int oscar_fields(oscar_handle h, int which, double *host_out, size_t n);

/* Same, into device memory (double) on the handle's stream; does not wait. */
int oscar_fields_device(oscar_handle h, int which, double *dev_out, size_t n);

/* Overwrite one state field from host memory (double): ALPHA (recomputes the
 * interface normals and curvature), U_VD, U_CR, P_VD (also selected by P),
 * P_CR, PHI_VD, PHI_CR. Waits for the stream. */
int oscar_set_field(oscar_handle h, int which, const double *host_in, size_t n);

/* Statistics of the instance (waits for the stream). */
int oscar_stats(oscar_handle h, oscar_stats_t *out);

/* Multigrid schedule and launch shape of an instance's pressure solves (not
 * part of the paper's method, whose solver is unnamed; these choose how fast
 * the same solves converge, not what they converge to, within cg_rtol).
 * Defaults at creation: {2, 2, 2, 1024, 8, 0, 1}. */
typedef struct {
    int mg_nu;          /* red-black Gauss-Seidel sweep pairs per smoothing step, finest level: 1..4 */
    int mg_nu_mid;      /* the same on the levels between the finest and the coarse CTA: 1..4 */
    int mg_nu_cta;      /* the same on the levels held by the single coarse CTA: 1..6 */
    int cta_cells;      /* levels of at most this many cells (and fitting its shared memory) go to the
                           coarse CTA: 1..1024 */
    int coarse_refresh; /* the coarsest CTA level's explicit inverse is formed on the first PISO set-up of
                           a step call and every coarse_refresh-th after it, kept in between: 1..1000 */
    int block_x;        /* cap on the x extent of the 256-thread blocks of cell kernels: 0 (none), 32, 64,
                           128 or 256 */
    int cta_global;     /* 1: the level just above the coarse CTA's levels (not the finest) is worked by
                           the same CTA, its x and b in shared memory and its coefficients read from
                           global memory, when that fits; 0: by per-level kernels */
} oscar_schedule;

/* Read the schedule of an instance. */
int oscar_get_schedule(oscar_handle h, oscar_schedule *out);

/* Replace the schedule (waits for the stream; the step graphs are rebuilt at
 * the next step call). OSCAR_E_INVALID_ARG for a value out of range, while an
 * asynchronous step is pending, or when the coarse levels chosen by cta_cells
 * do not fit the coarse CTA's shared memory; the schedule is then unchanged. */
int oscar_set_schedule(oscar_handle h, const oscar_schedule *s);

/* Release all device memory of the instance. */
int oscar_destroy(oscar_handle h);

/* Static string for a return code. */
const char *oscar_strerror(int code);

/* In-step kernel timing (measurement support, not part of the method).
 * enable = 1 clears any previous recording and makes the following step calls
 * run their launch sequence eagerly (host-driven loops with one control-word
 * read-back per loop trip, instead of the captured graphs), with a pair of
 * CUDA events on the handle's stream around every kernel launch; the device
 * times are accumulated per (kernel function, launch grid size), so that a
 * multigrid kernel on two levels gives two entries. enable = 0 stops and keeps
 * the recording. The numerics of a profiled step are those of the graph step
 * (same kernels in the same order). Errors: OSCAR_E_INVALID_ARG while an
 * asynchronous step is pending; OSCAR_E_CUDA if events cannot be created. */
int oscar_profile(oscar_handle h, int enable);

/* Entry `index` of the recording: *count_out (may be NULL) receives the number
 * of entries; name_out (may be NULL) receives up to name_cap - 1 characters of
 * the kernel's (mangled) name; grid_out the blocks of its launches; total_ms the
 * summed device time [ms]; launches the number of timed launches. Waits for
 * the handle's stream. Returns OSCAR_E_INVALID_ARG when index >= the count
 * (count_out is still written). */
int oscar_profile_read(oscar_handle h, int index, int *count_out, char *name_out, size_t name_cap,
                       unsigned *grid_out, double *total_ms, long long *launches);

/* In-graph kernel timing by difference (measurement support, not part of the
 * method). enable = 1 makes the following step calls issue every finest-level
 * red-black half sweep that is not fused with a dot product twice in a row:
 * a half sweep reads only the other colour, so the repeat writes the values
 * just written and the fields stay bitwise those of a normal step. The steps
 * run from their (rebuilt) CUDA graphs as usual; the time they add over the
 * same steps of an identical instance, divided by the launches they add
 * (oscar_stats kernel_launches), is the in-graph duration of one such sweep
 * with its operands where the step leaves them. enable = 0 restores normal
 * steps. Waits for the stream. OSCAR_E_INVALID_ARG while an asynchronous step
 * is pending. */
int oscar_profile_repeat(oscar_handle h, int enable);

/* Phase volume sum over fluid cells of alpha * cell_volume, computed without
 * allocating any device memory. The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc, such as code running while
 * a stream is being captured into a CUDA graph, or hosts that give the GPU a
 * fixed memory budget and forbid later allocation.
 *   alpha_dev   device double[ncell] (values in solid cells are ignored)
 *   solid_dev   device uint8[ncell], 1 = solid
 *   ncell       1 .. 16,777,216 cells; larger grids return OSCAR_E_INVALID_ARG
 *   result_dev  device double[1] receiving the volume
 *   stream      cudaStream_t of the call (NULL = default stream)
 * Scratch: a 512 KiB static device array inside the library image, held by
 * every GPU that loads the library until the process exits. The first call on
 * a device looks up that array's device address and clears it (once per
 * device, with that device current, thread-safe; it waits for the clear on
 * the given stream); make that first call before any stream capture. The
 * looked-up address belongs to the device's context: do not call this again
 * in a process after cudaDeviceReset. The result is not waited for. Every call shares the scratch, which keeps the
 * last call's contents: calls that may overlap on the GPU (different streams,
 * no ordering between them) race and must not be issued. */
int oscar_phase_volume_noalloc(const double *alpha_dev, const uint8_t *solid_dev, long long ncell,
                               double cell_volume, double *result_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* OSCAR_H */
