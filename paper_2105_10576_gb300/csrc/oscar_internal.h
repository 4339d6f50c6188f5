// Host-side instance layout shared by the C-ABI unit and the per-precision
// solver units. Device code lives in oscar_kernels.cuh.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <vector>

#include "../../include/oscar.h"

namespace oscar {

constexpr int kMaxLevels = 24;
constexpr int kRedBlocks = 1216;      // 152 SMs x 8: fixed grid of every reduction (deterministic order)
constexpr int kRedSlots = 16;         // partial-sum slots
constexpr double kSyncTimeoutSec = 600.0;
constexpr size_t kCtaImageBytes = 224 * 1024;   // shared-memory budget of the coarse CTA

// Scalar slots in the device scalar array (double).
enum Slot {
    S_BB = 0, S_RR, S_RZ0, S_RZ1, S_PAP, S_QSUM, S_RES, S_NRM, S_DUMAX, S_VOL, S_TARGET, S_E, S_DU, S_TEST,
    S_ITARGET, S_ALPHA, S_BETA, S_ALPHA_F, S_BETA_F, S_TMP, S_AREA0, S_AREA1, S_COUNT
};

// Integer control words on the device (relaxation and PCG loop state).
enum Ctl { C_K = 0, C_N, C_IT, C_ITSUM, C_NAN, C_NOTCONV, C_COND, C_OUT, C_OSUM, C_PACK, C_COUNT = 12 };

// One captured and instantiated step graph.
struct GraphSlot {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    double dt;
    int valid;
    long long n_pre;    // kernels outside every loop body
    long long n_body;   // kernels per relaxation sub-step outside the PCG bodies
};

struct GridH {
    int dim, nx, ny, nz, ncell;
    int nf[3];
    double h[3], S[3], V;
};

struct Level {
    GridH g;
    int r[3];            // coarsening ratio to the next level (1 or 2 per direction)
    uint8_t *fluid;      // level >= 1: any fine child fluid
    void *c[3];          // face coefficients (T)
    void *diag;          // T
    void *idiag;         // T: 1 / diag on fluid cells, else 0
    void *x, *b, *res;   // T
};

// In-step kernel timing: while enabled, step calls run their launch sequence
// eagerly (host-driven loops instead of graphs) with a pair of CUDA events on
// the launching stream around every kernel, accumulated per kernel function
// and launch geometry (a multigrid kernel on two levels is two entries).
constexpr int kProfPool = 8192;
constexpr int kProfKinds = 192;
struct ProfEntry {
    const void *fn;
    unsigned grid, block;
    double total_ms;
    long long launches;
};
struct Profiler {
    int enabled;
    int created;
    int n;                       // event pairs in use
    long long dropped;
    int slot_entry[kProfPool];
    cudaEvent_t ev0[kProfPool], ev1[kProfPool];
    int nent;
    ProfEntry ent[kProfKinds];
};
// the profiler of the step being issued on this host thread (null when off)
inline thread_local Profiler *t_prof = nullptr;
// cap on the x extent of the thread blocks of cell kernels (0: no cap) of the
// instance whose launches this host thread is issuing (schedule block_x)
inline thread_local int t_block_x = 0;
struct BlockXScope {
    int saved;
    explicit BlockXScope(int v) : saved(t_block_x) { t_block_x = v; }
    ~BlockXScope() { t_block_x = saved; }
};
int prof_begin(Profiler *P, cudaStream_t st, const void *fn, dim3 grid, dim3 block);
void prof_end(Profiler *P, cudaStream_t st, int slot);
int prof_drain(Profiler *P, cudaStream_t st);

// Device memory of one instance; element type T (double or float) is fixed by
// the precision chosen at creation. CG vectors and accumulators are double.
struct Instance {
    oscar_params P;
    GridH g;
    cudaStream_t stream;
    int prec;
    long long n_fluid;
    double cos_theta, deltaN;

    // arena
    void *arena;
    size_t arena_bytes;

    uint32_t *info;        // per-cell face types + fluid flag
    // cell fields (T)
    void *alpha, *alpha_new, *alpha_s, *alpha_tmp, *kappa;
    void *aL, *Pp, *Pm, *Rp, *Rm;
    void *rA;
    void *hbya[3], *vold[3], *u_vd[3], *u_cr[3], *G[9];
    // cell fields (double)
    double *u_sum[3], *p_vd, *p_cr;
    double *cg_b, *cg_r, *cg_z, *cg_p, *cg_Ap;   // Krylov vectors hold T on the mixed path
    void *cg_e;            // mixed path: correction of the outer defect-correction step (T)
    double *cg_r64;        // mixed path: FP64 residual b - M q of the outer defect correction
    // FP64 pressure operator: level-0 face coefficients in FP64 (the mixed
    // path keeps copies; the FP64 path points at level 0's arrays)
    double *cf64[3];
    // face fields (T)
    void *nf[3], *phi_vd[3], *phi_cr[3], *phic[3], *phis[3], *fst[3];
    // multigrid (level 0 coefficients are the pressure operator's)
    int nlev;
    Level lev[kMaxLevels];
    // reductions
    double *partials;      // kRedSlots * red_stride
    int red_stride;        // partials per slot: max(kRedBlocks, blocks of a cell launch)
    int lc0;               // first multigrid level solved by the single-CTA coarse kernel
    size_t cta_smem;       // shared memory of the coarse kernel
    size_t cta_img_bytes;  // bytes of the coarse levels' image (the start of that shared memory)
    int lg;                // level worked by the coarse CTA with global coefficients, -1 when none
    void *cta_img;         // shared-memory image of the coarse levels (kCtaImageBytes, built per PISO set-up)
    int pending;           // kind (0 drag, 1 relax, 2 standard) of a launched step not yet waited for, or -1
    double pending_dt;
    int pending_N;
    unsigned *ticket;      // block counter of the single-pass reductions (0 between kernels)
    double *scal;          // S_COUNT device scalars
    double *scal_host;     // pinned mirror
    double *stage_host;    // pinned staging for field transfers (max(ncell, faces) doubles)
    double *stage_dev;     // device staging of the same length
    size_t stage_len;

    // statistics
    int last_kf, last_N;
    double last_E, last_dU;
    long long cg_iters_total;
    int cg_iters_last;
    long long cell_updates;
    int mg_nu, mg_nu_c, mg_coarse_sweeps;   // sweeps on the finest level, on coarser levels, on the coarsest
    int mg_nu_cta;         // sweeps on the levels held by the coarse CTA
    int repeat_fine;       // measurement: finest-level plain half sweeps issued twice (oscar_profile_repeat)
    int coarse_refresh;    // the coarsest level's inverse is formed every this many PISO set-ups
    int cta_cells;         // levels of at most this many cells go to the coarse CTA
    int block_x;           // cap on the x extent of cell-kernel blocks (0: none)
    int cta_global;        // 1: the level above the CTA's may go to the CTA with global coefficients
    long long nlaunch;     // kernel launches issued by the host (eager or into a capture)
    long long nexec;       // kernels executed on the device (graph executions counted by loop trips)
    Profiler *prof;
    // graphs: 0 drag step, 1 relaxation, 2 standard step
    GraphSlot gslot[3];
    cudaStream_t side[4];  // capture streams of nested loop bodies
    int depth;             // current nesting depth while capturing
    int capturing;
    long long n_cg_body;   // kernels per PCG iteration
    long long n_outer_body; // kernels per defect-correction trip outside the PCG body
    long long cg_bodies_captured;
    int *ctl;              // device control words
    int *ctl_host;         // pinned: initial control words (read by the graph) and read-back
    double last_dt;
    int eager;             // 1: host-driven loops, no graphs (for per-kernel profiling)
    int own_stream;        // the library created I.stream
};


// per-precision entry points (defined in oscar_kernels.cuh, instantiated twice)
template <typename T> struct Solver {
    static int setup(Instance &I, const uint8_t *solid_dev, const double *alpha0_dev);
    static int drag_step(Instance &I, double dt);
    static int relax(Instance &I, double dt, int N, int *kf, double *test);
    static int standard_step(Instance &I, double dt);
    static int launch_step(Instance &I, int kind, double dt, int N);   // no wait
    static int finish_step(Instance &I, int *kf, double *test);       // waits for the launched step
    static int field_to_device(Instance &I, int which, double *dst, size_t n);
    static int field_from_device(Instance &I, int which, const double *src, size_t n);
    static int phase_volume(Instance &I, double *out);
    static void release_graphs(Instance &I);
    static int choose_cta(Instance &I, long long cap);   // first CTA level and its shared memory
};

int sync_bounded(cudaStream_t s, double timeout_sec);
size_t field_len(const Instance &I, int which);

}  // namespace oscar
