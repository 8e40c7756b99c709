/*
 * sgpic.h -- C ABI of the GB300 sparse-grid combination-technique PIC library.
 *
 * The library advances electrostatic particle-in-cell runs whose charge
 * density and field are represented by the truncated sparse-grid
 * combination technique of Muralikrishnan, Cerfon, Frey, Ricketson and
 * Adelmann, "Sparse grids based adaptive noise reduction strategy for
 * particle-in-cell schemes" (arXiv:2008.09441).  One step is:
 *
 *   cell-key sort of the particles (every `sort_every` steps)
 *   -> CIC deposit onto every component grid (Section 4.1, eq. restriction,
 *      computed through the regular grid as Proposition 1 allows)
 *   -> spectral Poisson solve on every component grid (Section 2)
 *   -> signed combination of the component fields on the regular nodes
 *      (eq. sparse_filter applied to the fields, coefficients of Section 4.2)
 *   -> CIC gather and leapfrog / Boris push (Section 2, steps 3-4).
 * sg_params.mode selects the paper's filter mode instead (eq. sparse_filter,
 * Algorithm 2): the regular-grid density is filtered by the same
 * combination and solved once on the regular grid.
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: SG_OK (0) or a negative SG_ERR_*
 *     code.  sg_strerror() names it; sg_last_error() gives the detail text of
 *     the most recent failure in the calling thread.  No C++ exception crosses
 *     this boundary.
 *   - Geometry: periodic box [0, L_1) x ... x [0, L_d), d in {2, 3}.  Particle
 *     positions are passed as fractions of the box, u_m = x_m / L_m (values
 *     outside [0, 1) are wrapped periodically).  Velocities are physical.
 *     Grids are node-centred by default (node k of a level-l axis at
 *     x = k L / 2^l) or cell-centred (x = (k + 1/2) L / 2^l, sg_params.centring);
 *     "regular nodes" below are the level-n nodes in either case.
 *   - Grid arrays are flat, x fastest: index = i_1 + 2^l_1 (i_2 + 2^l_2 i_3).
 *   - Particle arrays are structure-of-arrays in the run's precision
 *     (float for SG_FP32, double for SG_FP64).
 *   - A handle is not thread safe: one thread at a time per handle.  All
 *     device work of a handle runs on its stream (params.stream, or a stream
 *     the library creates when that is NULL).
 *   - Inputs are copied; the caller keeps ownership of every buffer it passes.
 */
#ifndef SGPIC_H
#define SGPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SG_OK 0
#define SG_ERR_INVALID (-1)     /* bad argument (NULL, out of range, non-finite input) */
#define SG_ERR_UNSUPPORTED (-2) /* valid request the library does not implement */
#define SG_ERR_OOM (-3)         /* device allocation failed */
#define SG_ERR_SIZE (-4)        /* caller buffer too small / size mismatch */
#define SG_ERR_TIMEOUT (-5)     /* a bounded wait expired */
#define SG_ERR_CUDA (-6)        /* CUDA runtime error (detail in sg_last_error) */
#define SG_ERR_RANGE (-7)       /* empty or invalid truncation-parameter range */
#define SG_ERR_NONFINITE (-8)   /* a kernel saw a non-finite particle state */
#define SG_ERR_STATE (-9)       /* call not valid in the handle's current state */

#define SG_FP32 0
#define SG_FP64 1

#define SG_TAU_ADAPTIVE (-1)          /* run Algorithm 1 (tauEstimator) every step */
#define SG_TAU_CONST_PAPER 0          /* eq. grid_constants + eq. particle_constant */
#define SG_TAU_CONST_EMPIRICAL 1      /* eq. empirical_constants */
#define SG_MODE_COMBINE 0
#define SG_MODE_FILTER 1
#define SG_NODE_CENTRED 0 /* node k of a level-l axis at x_k = k L / 2^l */
#define SG_CELL_CENTRED 1 /* node k at the cell centre x_k = (k + 1/2) L / 2^l */
#define SG_COMBINE_FLOAT_FLOAT 0 /* FP32 path: combination in float pairs (about 48 bits) */
#define SG_COMBINE_FP64 1        /* FP32 path: combination accumulated in double */

typedef struct sg_pic sg_pic; /* opaque run handle; owns all its device memory */

typedef struct {
  int dim;      /* 2 or 3 */
  double L[3];  /* box lengths L_m > 0 (L[2] ignored in 2D) */
} sg_domain;

typedef struct {
  size_t n;          /* number of particles */
  int on_device;     /* 1: pointers are device memory; 0: host memory */
  const void* u[3];  /* positions as fractions of L_m, one array per axis */
  const void* v[3];  /* velocities, one array per axis */
  const void* w;     /* per-particle charge q_p; mass is q_p / qm */
} sg_particles;

typedef struct {
  size_t n;
  int on_device;
  void* u[3];
  void* v[3];
  void* w;
} sg_particles_out;

typedef struct {
  int precision;      /* SG_FP32 or SG_FP64: particles, deposit, solves */
  int tau;            /* truncation parameter 1..n, or SG_TAU_ADAPTIVE */
  double dt;          /* time step */
  double qm;          /* charge-to-mass ratio q/m (-1 in the paper, Section 5) */
  double B[3];        /* uniform external magnetic field (Boris push if nonzero;
                         in 2D only B[2] is allowed) */
  double Eext_lin[3]; /* external field E_m = Eext_lin[m] (x_m - L_m/2) */
  double alpha;       /* denoising threshold fraction (Section 4.3.3) */
  double pc_ref;      /* reference particles per cell (P_c)_ref (Section 4.3.3) */
  int tau_constants;  /* SG_TAU_CONST_PAPER or SG_TAU_CONST_EMPIRICAL */
  int sort_every;     /* cell-key sort period in steps; 0 = library default (4 in 2D, 6 in 3D) */
  void* stream;       /* cudaStream_t for all work of the run; NULL = own stream */
  int mode;           /* SG_MODE_COMBINE (0): sparse PIC, a spectral solve on every
                         component grid and the signed combination of their fields
                         (Section 4.1); SG_MODE_FILTER (1): the paper's filter mode
                         (eq. sparse_filter, Algorithm 2): the regular-grid density
                         is filtered, rho_f = sum_i c_i P_i R_i rho~, and solved
                         once on the regular grid.  Either way the push gathers
                         from a field on the regular nodes. */
  int centring;       /* SG_NODE_CENTRED (0): nodes at x_k = k h, where Proposition 1
                         makes the two-step deposit the direct one; SG_CELL_CENTRED
                         (1): nodes at cell centres (the paper's choice, Section 4.3),
                         component densities R_i rho~ with the two-step shape W_c of
                         Appendix A, and the gather through the same shape (P_i to
                         the regular grid, then CIC).  Any other value:
                         SG_ERR_INVALID. */
  int combine;        /* accumulation of the signed combination of the component
                         fields (Section 4.1, coefficients of Section 4.2) on the
                         FP32 path: SG_COMBINE_FLOAT_FLOAT (0, default) sums every
                         term with an error-free float addition whose error is
                         carried in a second float; SG_COMBINE_FP64 (1) forms each
                         term and the sum in double (slower on GB300, whose double
                         rate is a small fraction of its float rate).  Either way
                         the result is stored as hi + lo floats and the field
                         energy is reduced in FP64.  The FP64 path always
                         accumulates in double.  Any other value: SG_ERR_INVALID. */
} sg_params;

typedef struct {
  long long step;               /* steps taken */
  double t;                     /* step * dt */
  int tau;                      /* truncation parameter in use */
  int n_grids;                  /* number of component grids */
  double charge_total;          /* sum_p q_p (FP64, from the particles) */
  double charge_combined;       /* sum_i c_i V_i sum_k rho_i(x_k) (FP64) */
  double charge_grid_max_abs_err; /* max_i |V_i sum_k rho_i - sum_p q_p| */
  double field_energy;          /* 0.5 h^d sum_j |E_comb(x_j)|^2 at time t */
  double field_energy_prev;     /* the same at time t - dt (0 before the first step) */
  double kinetic_energy;        /* 0.5 sum_p m_p v^{-1/2}.v^{+1/2}, time-centred at t - dt */
  unsigned long long count_checksum; /* sum_p (key_p + 1) mod 2^64 at the last sort */
} sg_diag;

/* ---- run lifecycle -------------------------------------------------------
 * sg_pic_init: create a run.  level_n: regular grid 2^n per axis
 * (Section 4.1); dim 2 or 3 (must equal domain->dim); shape_order must be 1
 * (CIC / linear, the paper's only shape, eq. restriction), else
 * SG_ERR_UNSUPPORTED.  Limits: 1 <= tau <= n; dim*n <= 24; 2 <= n.
 * Copies the particles (host or device), wraps positions into [0,1), sorts
 * by cell key, deposits, solves and takes the backward half kick
 * v^{-1/2} = v^0 - (q/m) E(x^0) dt/2 (Boris form when B != 0).
 * On success *out owns every device buffer of the run. */
int sg_pic_init(const sg_domain* domain, int level_n, int dim, int shape_order,
                const sg_particles* particles, const sg_params* params, sg_pic** out);

/* Advance nsteps >= 0 steps (asynchronous on the run's stream; graph replay). */
int sg_pic_step(sg_pic* h, int nsteps);

/* Synchronise the run's stream and return its FP64 diagnostics. */
int sg_pic_diagnostics(sg_pic* h, sg_diag* out);

/* Pipelined diagnostics, for monitoring a run without stalling its stream.
 * sg_pic_diagnostics_post enqueues on the run's stream the read-back of the
 * FP64 diagnostics as they stand after every step launched so far, into one
 * of SG_DIAG_RING pinned host slots owned by the run, and returns without
 * waiting.  sg_pic_diagnostics_collect waits for the OLDEST posted record and
 * returns it: the values sg_pic_diagnostics would have returned at that post
 * (step, tau and grid set included, even if sg_pic_set_tau changed them since).
 * Errors: post with SG_DIAG_RING records pending, or collect with none, gives
 * SG_ERR_STATE; collect gives SG_ERR_NONFINITE (with *out filled) when the
 * record saw a non-finite particle state.  sg_pic_destroy drops records
 * left pending.  sg_pic_diagnostics may be called in between; it does not
 * touch the slots. */
#define SG_DIAG_RING 4
int sg_pic_diagnostics_post(sg_pic* h);
int sg_pic_diagnostics_collect(sg_pic* h, sg_diag* out);

/* Algorithm 1 (tauEstimator, Section 4.3.3) on the current regular-grid
 * density: FFT, hard threshold (eq. denoising) with
 * eps = alpha sqrt(pc_ref / P_c) max|rho^|, constants (params.tau_constants),
 * then grid error + particle noise (eq. 2D/3D_grid_error, 2D/3D_particle_noise)
 * for tau in [1, n-3] (2D) or [1, n-2] (3D); returns the argmin (ties: the
 * smallest tau).  est_grid / est_noise (may be NULL) receive the estimates for
 * tau = 1..cap.  Computed in FP64 on the GPU.  SG_ERR_RANGE if the range is
 * empty; SG_ERR_UNSUPPORTED for non-cubic boxes (the estimates assume one L).
 * Does not change the run's tau. */
int sg_pic_select_tau(sg_pic* h, int* tau, double* est_grid, double* est_noise, int cap);

/* Switch the truncation parameter (1..n) for the following steps: rebuilds
 * the component-grid set and re-deposits / re-solves the current state. */
int sg_pic_set_tau(sg_pic* h, int tau);

/* Copy particle states to caller buffers in the ORIGINAL particle order
 * (the order given at init), whatever sorts happened since.  out->n must
 * equal the run's particle count; buffers are host or device per on_device. */
int sg_pic_get_particles(sg_pic* h, const sg_particles_out* out);

/* Cell keys (Morton order of the level-n cell, x lowest bit) of the particles
 * in their current storage order, and per-cell counts indexed by key.
 * Recomputes both from the current positions; cap_* are element capacities
 * (keys: n particles, counts: 2^(d n)); either pointer may be NULL.  Host
 * buffers. */
int sg_pic_get_keys(sg_pic* h, uint32_t* keys, uint32_t* counts, size_t cap_keys, size_t cap_counts);

/* Combined field E_comb = sum_i c_i P_i E_i on the regular nodes, FP64,
 * component-major: out[m * 2^(d n) + node].  Host buffer, cap in doubles. */
int sg_pic_get_field(sg_pic* h, double* E, size_t cap);

/* Component-grid charge densities rho_i, concatenated in grid order
 * (sg_pic_get_grids), FP64, host buffer, cap in doubles. */
int sg_pic_get_grid_charge(sg_pic* h, double* rho, size_t cap);

/* Component fields E_i: for each grid in order, d blocks of 2^|l_i| values
 * (E_1 block, E_2 block, ...).  FP64 host buffer, cap in doubles.
 * SG_ERR_STATE in SG_MODE_FILTER (no component fields are solved). */
int sg_pic_get_grid_field(sg_pic* h, double* E, size_t cap);

/* Regular-grid charge density rho~ of the current positions (the tau = n
 * deposit used by Algorithm 1), FP64 host buffer of 2^(d n) values. */
int sg_pic_get_regular_charge(sg_pic* h, double* rho, size_t cap);

/* The charge density the field comes from, on the regular nodes (FP64 host
 * buffer of 2^(d n) values): sum_i c_i P_i rho_i, the sparse-grid density of
 * eq. sparse_filter (Section 4.1) -- in SG_MODE_FILTER the filtered density
 * its regular-grid solve used, in SG_MODE_COMBINE the same combination of
 * the component densities (whose fields the run combines). */
int sg_pic_get_density(sg_pic* h, double* rho, size_t cap);

/* Grid set in use: *n_grids receives the count; levels (3 ints per grid,
 * unused axes 0) and coeffs receive up to cap grids. */
int sg_pic_get_grids(sg_pic* h, int* n_grids, int* levels, int* coeffs, int cap);

/* Checkpoint: *size receives the byte size; with buf != NULL and *size large
 * enough, writes the full run state (particles in original order, step, tau,
 * time-centring).  sg_pic_load restores it into a run created with the same
 * domain, level, dimension, precision, particle count, mode and centring;
 * otherwise SG_ERR_INVALID. */
int sg_pic_save(sg_pic* h, void* buf, size_t* size);
int sg_pic_load(sg_pic* h, const void* buf, size_t size);

/* Device pointers of the run's state for callers that chain their own
 * kernels (valid until the next sort / destroy): u[d], v[d], w arrays in the
 * current storage order. */
int sg_pic_device_particles(sg_pic* h, sg_particles_out* out);

/* Count of library kernels launched on this handle so far (graph replays
 * count each kernel node). */
int sg_pic_kernel_launches(sg_pic* h, unsigned long long* count);

/* Device-event timing of the run's last sg_pic_step call, per stage
 * (0 gather-push, 1 sort, 2 deposit, 3 restrict, 4 solve, 5 combine) in
 * milliseconds, summed over that call's steps; in SG_MODE_FILTER entry 4 is
 * the density filter (sum_i c_i P_i R_i) and entry 5 the regular-grid solve.  Enabled with
 * sg_pic_set_profiling(h, 1), which replaces graph replay by direct launches
 * with events between the stages while on.  With cap >= 9, entries 6..8
 * report the init-time autotuner: the solve variant in use (0 per-axis
 * passes, 1 one block per grid) and the two timings (ms) it compared; with
 * cap >= 10 entry 9 is 1 when those timings came from an earlier run of the
 * same precision, dimension, level and tau in this process (the tuner's
 * cache), 0 when this run measured them.  With cap >= 21, entries 10..20
 * report the particle-pass tuner, which times, on the run's own particles
 * at init, the push with half, one and two resident waves of blocks (the
 * particles per block; a zero time step, which leaves every particle as it
 * is) and the deposit with windows of 4096, 6144, 8192 and 12288 nodes of
 * 64-bit capacity (the window's side and the windows per SM), and keeps
 * the defaults (one wave, 8192) unless a candidate is 3% faster: 10 push
 * blocks in use, 11 blocks of one resident wave, 12..14 the three push
 * timings, 15 the window capacity in use, 16..19 the four deposit timings,
 * 20 whether they came from an earlier run of the same shape (precision,
 * dimension, level, log2 of the particle count, centring, push kind).
 * Just before the run's first sort step (particles drifted for a whole sort
 * period) the four deposit windows are timed again and the window with the
 * smallest sum of the two timings is kept (3% rule; a change re-captures
 * the step graphs); with cap >= 25, entries 21..24 hold those timings (0
 * before that step, or when the cache held a refined choice).  Runs created
 * with sg_pic_init_deferred keep the defaults. */
int sg_pic_set_profiling(sg_pic* h, int on);
int sg_pic_stage_times(sg_pic* h, double* ms, int cap);

/* Solve variant of the combination mode: SG_SOLVE_AUTO (-1, the default:
 * both variants timed at init and at every grid-set change, the faster
 * kept), SG_SOLVE_PASSES (0: batched FFT passes per axis over all
 * component grids) or SG_SOLVE_ONE_BLOCK (1: one block solves one whole
 * component grid in shared memory).  Both compute the same fields.  A fixed
 * variant stays through later grid-set changes.  Returns SG_ERR_INVALID for
 * another value and SG_ERR_UNSUPPORTED for SG_SOLVE_ONE_BLOCK when a
 * component grid exceeds the one-block size; synchronises the run's
 * stream.  No effect on the filter mode's regular-grid solve, nor on the
 * cross-run solve of batched serving, which always takes one block per
 * (run, grid). */
#define SG_SOLVE_AUTO (-1)
#define SG_SOLVE_PASSES 0
#define SG_SOLVE_ONE_BLOCK 1
int sg_pic_set_solve_variant(sg_pic* h, int variant);

void sg_pic_destroy(sg_pic* h);

const char* sg_strerror(int status);
const char* sg_last_error(void);
const char* sg_version(void);

/* ---- host-only helpers (no GPU and no CUDA call) --------------------------
 * sg_combination_grids: the component grids of the truncated combination
 * technique (Section 4.2) for dim in {2, 3}, level n and truncation tau:
 * every level vector l with tau <= l_m <= n and |l|_1 = n + (dim-1) tau - q,
 * coefficient (-1)^q C(dim-1, q), q = 0..dim-1, in the order the library
 * uses (q ascending, then lexicographic with the last axis fastest).
 * *count receives the number of grids.  With levels and coeffs non-NULL and
 * cap >= *count, levels[3 i + m] receives l_m of grid i (0 for m >= dim) and
 * coeffs[i] its coefficient.  SG_ERR_INVALID for dim outside {2, 3}, n < 1,
 * tau outside [1, n] or a NULL count; SG_ERR_SIZE when cap is too small
 * (*count is still written). */
int sg_combination_grids(int dim, int n, int tau, int* levels, int* coeffs, int cap, int* count);
/* sg_estimate_footprint: the device bytes a run of these sizes allocates, as
 * the serving layer's admission control estimates them (an upper estimate).
 * SG_ERR_INVALID for a bad precision, dim, n or tau, or a NULL bytes. */
int sg_estimate_footprint(int precision, int dim, int n, int tau, size_t n_particles, size_t* bytes);

/* ---- cell-key sort as a stand-alone operation ----------------------------
 * sg_cell_sort: keys (Morton order of floor(u_m 2^level)), a stable sort
 * permutation and per-cell counts of n positions u (device pointers,
 * precision SG_FP32 or SG_FP64, dim arrays).  Outputs (device): keys_sorted
 * (n), perm (n: sorted position -> input index), counts (2^(dim*level)).
 * Scratch is allocated and freed inside the call.  stream may be NULL. */
int sg_cell_sort(int precision, int dim, int level, size_t n, const void* const* u,
                 uint32_t* keys_sorted, uint32_t* perm, uint32_t* counts, void* stream);

/* sg_cell_sort_static: the same sort, with the same arguments and results,
 * for callers that must not allocate device memory -- for example code that
 * runs under a device-memory budget owned by another allocator, or loops
 * where an allocation or free could synchronise the device or fail under
 * fragmentation.  (An engineering addition; the paper has no counterpart.)
 * Its scratch is a fixed array of SG_CELL_SORT_STATIC_WORDS 32-bit words
 * (about 3.2 MB) inside the library image, present on every GPU that loads
 * the library until the process exits; no call allocates or frees device
 * memory.  At most SG_CELL_SORT_STATIC_MAX positions: larger n returns
 * SG_ERR_SIZE without doing any work.  The first call on a device looks up
 * the array's device address with that device current (make that first call
 * before any stream capture on the device).  All calls share the array:
 * calls whose work can overlap on the GPU (different streams without
 * ordering) race and must be serialised by the caller. */
#define SG_CELL_SORT_STATIC_MAX 262144
#define SG_CELL_SORT_STATIC_WORDS 803072
int sg_cell_sort_static(int precision, int dim, int level, size_t n, const void* const* u,
                        uint32_t* keys_sorted, uint32_t* perm, uint32_t* counts, void* stream);

/* ---- sharded runs: one run's particles split over several handles --------
 * The particles of one run may be divided among several handles (one per
 * GPU, or several on one GPU), each holding its part.  The regular-grid
 * density is the only quantity the parts exchange: a step's deposit of each
 * part (the deposit the paper's Algorithm 2 sums over processes with one
 * MPI_Allreduce per component grid, Section 4.4) is summed over the parts
 * into every part's density, after which each part restricts, solves and
 * combines the same fields redundantly and pushes its own particles.
 *
 * sg_pic_init_deferred takes the arguments of sg_pic_init for this part's
 * particles and stops after depositing them: no field, no backward half
 * kick.  The caller then sums the densities (sg_pic_density_copy out, a sum
 * over the parts, sg_pic_density_copy in), sets the whole run's charge with
 * sg_pic_set_charge_total and calls sg_pic_start, which computes the fields
 * of the summed density and applies the half kick.  Each step is then
 * sg_pic_step_deposit, the same exchange, sg_pic_step_fields (sg_pic_step
 * on such a handle does no exchange).  Adaptive tau is not supported on a
 * deferred handle (SG_ERR_UNSUPPORTED: the estimator needs the whole run's
 * particle count).  Diagnostics of a part: the field energy and the grid
 * charges are the whole run's; the kinetic energy and the count checksum
 * are the part's own (sum them over the parts).  Calls out of order return
 * SG_ERR_STATE. */
int sg_pic_init_deferred(const sg_domain* domain, int level_n, int dim, int shape_order,
                         const sg_particles* particles, const sg_params* params, sg_pic** out);
int sg_pic_start(sg_pic* h);
/* First half of a step: push of this part's particles, the sort when due,
 * their deposit on the regular grid. */
int sg_pic_step_deposit(sg_pic* h);
/* Second half: restriction, component solves and combination (or the filter
 * mode's field) of the regular-grid density as it stands; completes the step. */
int sg_pic_step_fields(sg_pic* h);
/* The whole run's sum_p q_p (FP64): the mean density every solve removes and
 * the reference of the charge diagnostics.  Defaults to this part's charge. */
int sg_pic_set_charge_total(sg_pic* h, double q_total);
/* Copy the regular-grid density (2^{dn} values of the run's precision, x
 * fastest) between the run and the caller's device buffer of n values:
 * to_run = 0 out of the run, 1 into it.  Synchronises the run's stream, so
 * the buffer is ready for (or free after) the caller's own stream. */
int sg_pic_density_copy(sg_pic* h, void* dev_buf, size_t n, int to_run);

/* ---- serving: independent runs admitted as memory allows -----------------
 * A server keeps many independent runs resident on one GPU and advances all
 * of them together.  In batched mode a tick forks every resident run onto
 * its own stream.  Runs of the combination mode with a fixed tau whose
 * component grids fit one block's shared memory (a solve of the one-block
 * kind) and at most 2^20 particles take their step in three parts (the
 * shared solve waits for the slowest of them; larger runs are not bound by
 * launch latency and keep their own solve): the run's cached graph up to its
 * solve (push, sort when due, deposit, restriction); ONE launch per
 * precision that solves the component grids of all of them, one block per
 * (run, grid), from a job table of the runs' arenas; the run's cached graph
 * of the combination.  Other runs replay their cached graph of the whole
 * step.  The runs' kernels overlap on the device, and no graph is captured
 * again when runs arrive or leave.  In plain mode the runs are stepped in
 * turn with direct launches and one solve launch per component grid.  Requests are admitted in arrival
 * order while their estimated device footprint fits hbm_budget_bytes and a
 * slot is free; finished runs retire and free their memory. */
typedef struct sg_server sg_server;

typedef struct {
  sg_domain domain;
  int level_n;
  int dim;
  sg_particles particles; /* host arrays are copied at submit time */
  sg_params params;       /* params.stream is ignored (the server's stream) */
  int nsteps;
} sg_request;

#define SG_REQ_QUEUED 0
#define SG_REQ_RUNNING 1
#define SG_REQ_DONE 2
#define SG_REQ_FAILED 3

#define SG_SERVE_BATCHED 0 /* cached per-run graphs on the runs' streams, one cross-run solve launch */
#define SG_SERVE_PLAIN 1   /* runs stepped in turn, direct launches, one solve launch per grid */

int sg_serve_create(size_t hbm_budget_bytes, int max_slots, sg_server** out);
/* Select how ticks advance the resident runs (default SG_SERVE_BATCHED). */
int sg_serve_set_mode(sg_server* s, int mode);
/* Queue a request (copies its particle arrays); returns a ticket. */
int sg_serve_submit(sg_server* s, const sg_request* req, unsigned long long* ticket);
/* Admit what fits, then advance every resident run by one step. *active
 * receives the number of resident runs after the call. */
int sg_serve_tick(sg_server* s, int* active);
/* State of a ticket and (when running or done) its latest diagnostics. */
int sg_serve_poll(sg_server* s, unsigned long long ticket, int* state, sg_diag* last);
/* Final particle state of a finished request (original order). */
int sg_serve_result(sg_server* s, unsigned long long ticket, const sg_particles_out* out);
/* Per-step latency percentiles (ms) over all steps served so far and
 * aggregate particle-steps per second of device time. */
/* Cross-run solves of the batched mode so far: the launches and the
 * component grids they solved (summed over the launches).  Either pointer
 * may be NULL. */
int sg_serve_solve_stats(sg_server* s, unsigned long long* launches, unsigned long long* grids);
int sg_serve_stats(sg_server* s, double* p50_ms, double* p99_ms, double* particle_steps_per_s,
                   unsigned long long* steps_served);
void sg_serve_destroy(sg_server* s);

#ifdef __cplusplus
}
#endif
#endif /* SGPIC_H */
