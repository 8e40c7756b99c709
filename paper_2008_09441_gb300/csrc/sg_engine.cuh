// Host runtime of one sparse-grid PIC run: device memory, the component-grid
// set and its job tables, the per-step launch sequence and its CUDA graphs.
#pragma once

#include <cmath>
#include <cstring>
#include <vector>

#include "sg_kernels.cuh"

namespace sg {

struct GridSpec {
  int l[3];
  int coeff;
};

// Truncated combination technique (Section 4.2): all level vectors with
// l_m >= tau and |l|_1 = n + (d-1) tau - q, coefficient (-1)^q C(d-1, q),
// q = 0..d-1.  Order: q ascending, then lexicographic with the last axis
// fastest.
std::vector<GridSpec> combination_grids(int d, int n, int tau);

struct EngineConfig {
  int dim = 2, n = 0, tau = 1, precision = SG_FP32;
  double L[3] = {1, 1, 1};
  double dt = 0, qm = -1;
  double B[3] = {0, 0, 0};
  double eext_lin[3] = {0, 0, 0};
  double alpha = 0.01, pc_ref = 5;
  int tau_constants = SG_TAU_CONST_PAPER;
  int sort_every = 0;
  int mode = SG_MODE_COMBINE;
  bool cell = false;  // cell-centred grids (nodes at (k + 1/2) h)
  bool combine_fp64 = false;  // FP32 path: combination accumulated in double (else float-float)
  bool deferred = false;      // init stops after the deposit; start() computes the fields
  // deposit window capacity in regular nodes with 64-bit accumulators (64 KB;
  // a 128 x 128 window of 32-bit fixed point in 2D, 24^3 in 3D): large enough
  // for a chunk's particles a few steps after a sort
  int win_cap = 8192;
};

class EngineBase {
 public:
  virtual ~EngineBase() {}
  virtual int init(const EngineConfig& cfg, const sg_particles* p, cudaStream_t stream) = 0;
  virtual int step(int nsteps) = 0;
  virtual int diagnostics(sg_diag* out) = 0;
  virtual int diagnostics_post() = 0;
  virtual int diagnostics_collect(sg_diag* out) = 0;
  virtual int select_tau(int* tau, double* est_grid, double* est_noise, int cap) = 0;
  virtual int set_tau(int tau) = 0;
  virtual int get_particles(const sg_particles_out* out) = 0;
  virtual int get_keys(uint32_t* keys, uint32_t* counts, size_t cap_keys, size_t cap_counts) = 0;
  virtual int get_field(double* E, size_t cap) = 0;
  virtual int get_grid_charge(double* rho, size_t cap) = 0;
  virtual int get_grid_field(double* E, size_t cap) = 0;
  virtual int get_regular_charge(double* rho, size_t cap) = 0;
  virtual int get_density(double* rho, size_t cap) = 0;
  virtual int get_grids(int* n_grids, int* levels, int* coeffs, int cap) = 0;
  virtual int save(void* buf, size_t* size) = 0;
  virtual int load(const void* buf, size_t size) = 0;
  virtual int device_particles(sg_particles_out* out) = 0;
  virtual int set_profiling(int on) = 0;
  virtual int set_solve_variant(int variant) = 0;
  virtual int stage_times(double* ms, int cap) = 0;
  virtual unsigned long long kernel_launches() const = 0;
  virtual size_t device_bytes() const = 0;
  virtual cudaStream_t stream() const = 0;
  virtual size_t n_particles() const = 0;
  virtual long long steps_done() const = 0;
  // Plain serving path: direct launches, one solve launch per component grid.
  virtual int step_plain() = 0;
  // sharded runs (one handle per part of a run's particles)
  virtual int start() = 0;
  virtual int step_deposit() = 0;
  virtual int step_fields() = 0;
  virtual int set_charge_total(double q) = 0;
  virtual int density_copy(void* dev_buf, size_t n, int to_run) = 0;
  // cross-run solve (batched serving): the step split around the component
  // solves; solve_jobs appends this run's jobs as raw SolveJob<real> bytes
  virtual bool solve_batchable() const = 0;
  virtual int real_bytes() const = 0;
  virtual int step_pre() = 0;
  virtual int solve_jobs(std::vector<unsigned char>& out, int* max_size, int* max_log) = 0;
  virtual int step_post() = 0;
};

EngineBase* make_engine(int precision, int dim);

// Estimated device footprint of a run (bytes), for admission control.
size_t estimate_footprint(int precision, int dim, int n, int tau, size_t np);

}  // namespace sg
