// C ABI entry points (include/sgpic.h): argument validation, error text,
// the stand-alone cell-key sort and the run handle.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "sg_engine.cuh"

namespace sg {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }
const char* last_error() { return g_err.c_str(); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

}  // namespace sg

struct sg_pic {
  sg::EngineBase* e = nullptr;
};

using namespace sg;

static int invalid(const char* msg) {
  set_error(msg);
  return SG_ERR_INVALID;
}

static bool is_fin(double x) { return std::isfinite(x); }

extern "C" {

const char* sg_version(void) { return "sgpic-gb300 1.0 (sm_103a)"; }

int sg_combination_grids(int dim, int n, int tau, int* levels, int* coeffs, int cap, int* count) {
  if (!count) return invalid("sg_combination_grids: count is NULL");
  if ((dim != 2 && dim != 3) || n < 1 || tau < 1 || tau > n || dim * n > 30)
    return invalid("sg_combination_grids: need dim in {2, 3} and 1 <= tau <= n");
  const std::vector<GridSpec> g = combination_grids(dim, n, tau);
  *count = (int)g.size();
  if (!levels || !coeffs) return SG_OK;
  if (cap < (int)g.size()) {
    set_error("sg_combination_grids: capacity below the grid count");
    return SG_ERR_SIZE;
  }
  for (size_t i = 0; i < g.size(); ++i) {
    for (int m = 0; m < 3; ++m) levels[3 * i + m] = m < dim ? g[i].l[m] : 0;
    coeffs[i] = g[i].coeff;
  }
  return SG_OK;
}

int sg_estimate_footprint(int precision, int dim, int n, int tau, size_t n_particles, size_t* bytes) {
  if (!bytes) return invalid("sg_estimate_footprint: bytes is NULL");
  if ((precision != SG_FP32 && precision != SG_FP64) || (dim != 2 && dim != 3) || n < 2 || dim * n > 24 ||
      tau < 1 || tau > n)
    return invalid("sg_estimate_footprint: bad precision, dim, level or tau");
  *bytes = estimate_footprint(precision, dim, n, tau, n_particles);
  return SG_OK;
}

const char* sg_strerror(int status) {
  switch (status) {
    case SG_OK: return "ok";
    case SG_ERR_INVALID: return "invalid argument";
    case SG_ERR_UNSUPPORTED: return "unsupported";
    case SG_ERR_OOM: return "out of device memory";
    case SG_ERR_SIZE: return "buffer size mismatch";
    case SG_ERR_TIMEOUT: return "timeout";
    case SG_ERR_CUDA: return "CUDA error";
    case SG_ERR_RANGE: return "empty truncation-parameter range";
    case SG_ERR_NONFINITE: return "non-finite particle state";
    case SG_ERR_STATE: return "invalid state";
    default: return "unknown status";
  }
}

const char* sg_last_error(void) { return last_error(); }

static int init_run(const sg_domain* domain, int level_n, int dim, int shape_order, const sg_particles* particles,
                    const sg_params* params, sg_pic** out, bool deferred) {
  if (!out) return invalid("sg_pic_init: out is NULL");
  *out = nullptr;
  if (!domain || !particles || !params) return invalid("sg_pic_init: NULL argument");
  if (dim != 2 && dim != 3) return invalid("sg_pic_init: dim must be 2 or 3");
  if (domain->dim != dim) return invalid("sg_pic_init: domain->dim differs from dim");
  if (shape_order != 1) {
    set_error("sg_pic_init: only shape_order 1 (CIC / linear) is defined by the method");
    return SG_ERR_UNSUPPORTED;
  }
  if (level_n < 2 || dim * level_n > 24) return invalid("sg_pic_init: need 2 <= n and dim*n <= 24");
  if (params->tau != SG_TAU_ADAPTIVE && (params->tau < 1 || params->tau > level_n))
    return invalid("sg_pic_init: tau must be in [1, n] or SG_TAU_ADAPTIVE");
  if (params->tau == SG_TAU_ADAPTIVE && (dim == 2 ? level_n - 3 : level_n - 2) < 1) {
    set_error("sg_pic_init: adaptive tau needs a non-empty range [1, n-3] (2D) / [1, n-2] (3D)");
    return SG_ERR_RANGE;
  }
  if (params->precision != SG_FP32 && params->precision != SG_FP64)
    return invalid("sg_pic_init: precision must be SG_FP32 or SG_FP64");
  for (int m = 0; m < dim; ++m)
    if (!(domain->L[m] > 0) || !is_fin(domain->L[m])) return invalid("sg_pic_init: box lengths must be positive");
  if (!is_fin(params->dt) || !is_fin(params->qm) || params->qm == 0.0)
    return invalid("sg_pic_init: dt and qm must be finite, qm nonzero");
  for (int m = 0; m < 3; ++m)
    if (!is_fin(params->B[m]) || !is_fin(params->Eext_lin[m])) return invalid("sg_pic_init: non-finite field");
  if (dim == 2 && (params->B[0] != 0.0 || params->B[1] != 0.0)) {
    set_error("sg_pic_init: in 2D only B[2] (out of plane) is supported");
    return SG_ERR_UNSUPPORTED;
  }
  if (particles->n > 0xFFFFFFF0ull) return invalid("sg_pic_init: too many particles (max 2^32 - 16)");
  if (params->tau_constants != SG_TAU_CONST_PAPER && params->tau_constants != SG_TAU_CONST_EMPIRICAL)
    return invalid("sg_pic_init: unknown tau_constants");
  if (params->sort_every < 0) return invalid("sg_pic_init: sort_every must be >= 0");

  EngineConfig cfg;
  cfg.dim = dim;
  cfg.n = level_n;
  cfg.tau = params->tau;
  cfg.precision = params->precision;
  for (int m = 0; m < 3; ++m) {
    cfg.L[m] = m < dim ? domain->L[m] : 1.0;
    cfg.B[m] = params->B[m];
    cfg.eext_lin[m] = params->Eext_lin[m];
  }
  cfg.dt = params->dt;
  cfg.qm = params->qm;
  cfg.alpha = params->alpha;
  cfg.pc_ref = params->pc_ref;
  cfg.tau_constants = params->tau_constants;
  cfg.sort_every = params->sort_every;
  if (params->mode != SG_MODE_COMBINE && params->mode != SG_MODE_FILTER)
    return invalid("sg_pic_init: mode must be SG_MODE_COMBINE or SG_MODE_FILTER");
  cfg.mode = params->mode;
  if (params->centring != SG_NODE_CENTRED && params->centring != SG_CELL_CENTRED)
    return invalid("sg_pic_init: centring must be SG_NODE_CENTRED or SG_CELL_CENTRED");
  cfg.cell = params->centring == SG_CELL_CENTRED;
  if (params->combine != SG_COMBINE_FLOAT_FLOAT && params->combine != SG_COMBINE_FP64)
    return invalid("sg_pic_init: combine must be SG_COMBINE_FLOAT_FLOAT or SG_COMBINE_FP64");
  cfg.combine_fp64 = params->combine == SG_COMBINE_FP64;
  cfg.deferred = deferred;

  sg_pic* h = new (std::nothrow) sg_pic;
  if (!h) return SG_ERR_OOM;
  h->e = make_engine(params->precision, dim);
  if (!h->e) {
    delete h;
    return SG_ERR_OOM;
  }
  int st = h->e->init(cfg, particles, (cudaStream_t)params->stream);
  if (st != SG_OK) {
    std::string keep = last_error();
    delete h->e;
    delete h;
    set_error(keep);
    return st;
  }
  *out = h;
  return SG_OK;
}

int sg_pic_init(const sg_domain* domain, int level_n, int dim, int shape_order, const sg_particles* particles,
                const sg_params* params, sg_pic** out) {
  return init_run(domain, level_n, dim, shape_order, particles, params, out, false);
}

int sg_pic_init_deferred(const sg_domain* domain, int level_n, int dim, int shape_order,
                         const sg_particles* particles, const sg_params* params, sg_pic** out) {
  return init_run(domain, level_n, dim, shape_order, particles, params, out, true);
}

#define SG_H(h)                                         \
  do {                                                  \
    if (!(h) || !(h)->e) return invalid("NULL handle"); \
  } while (0)

int sg_pic_step(sg_pic* h, int nsteps) {
  SG_H(h);
  return h->e->step(nsteps);
}

int sg_pic_start(sg_pic* h) {
  SG_H(h);
  return h->e->start();
}

int sg_pic_step_deposit(sg_pic* h) {
  SG_H(h);
  return h->e->step_deposit();
}

int sg_pic_step_fields(sg_pic* h) {
  SG_H(h);
  return h->e->step_fields();
}

int sg_pic_set_charge_total(sg_pic* h, double q_total) {
  SG_H(h);
  return h->e->set_charge_total(q_total);
}

int sg_pic_density_copy(sg_pic* h, void* dev_buf, size_t n, int to_run) {
  SG_H(h);
  if (to_run != 0 && to_run != 1) return invalid("sg_pic_density_copy: to_run must be 0 or 1");
  return h->e->density_copy(dev_buf, n, to_run);
}

int sg_pic_diagnostics(sg_pic* h, sg_diag* out) {
  SG_H(h);
  if (!out) return invalid("sg_pic_diagnostics: out is NULL");
  return h->e->diagnostics(out);
}

int sg_pic_diagnostics_post(sg_pic* h) {
  SG_H(h);
  return h->e->diagnostics_post();
}

int sg_pic_diagnostics_collect(sg_pic* h, sg_diag* out) {
  SG_H(h);
  if (!out) return invalid("sg_pic_diagnostics_collect: out is NULL");
  return h->e->diagnostics_collect(out);
}

int sg_pic_select_tau(sg_pic* h, int* tau, double* est_grid, double* est_noise, int cap) {
  SG_H(h);
  if (!tau) return invalid("sg_pic_select_tau: tau is NULL");
  if (cap < 0) return invalid("sg_pic_select_tau: cap < 0");
  return h->e->select_tau(tau, est_grid, est_noise, cap);
}

int sg_pic_set_tau(sg_pic* h, int tau) {
  SG_H(h);
  return h->e->set_tau(tau);
}

int sg_pic_get_particles(sg_pic* h, const sg_particles_out* out) {
  SG_H(h);
  return h->e->get_particles(out);
}

int sg_pic_get_keys(sg_pic* h, uint32_t* keys, uint32_t* counts, size_t cap_keys, size_t cap_counts) {
  SG_H(h);
  return h->e->get_keys(keys, counts, cap_keys, cap_counts);
}

int sg_pic_get_field(sg_pic* h, double* E, size_t cap) {
  SG_H(h);
  if (!E) return invalid("sg_pic_get_field: NULL buffer");
  return h->e->get_field(E, cap);
}

int sg_pic_get_grid_charge(sg_pic* h, double* rho, size_t cap) {
  SG_H(h);
  if (!rho) return invalid("sg_pic_get_grid_charge: NULL buffer");
  return h->e->get_grid_charge(rho, cap);
}

int sg_pic_get_grid_field(sg_pic* h, double* E, size_t cap) {
  SG_H(h);
  if (!E) return invalid("sg_pic_get_grid_field: NULL buffer");
  return h->e->get_grid_field(E, cap);
}

int sg_pic_get_regular_charge(sg_pic* h, double* rho, size_t cap) {
  SG_H(h);
  if (!rho) return invalid("sg_pic_get_regular_charge: NULL buffer");
  return h->e->get_regular_charge(rho, cap);
}

int sg_pic_get_density(sg_pic* h, double* rho, size_t cap) {
  SG_H(h);
  if (!rho) return invalid("sg_pic_get_density: NULL buffer");
  return h->e->get_density(rho, cap);
}

int sg_pic_get_grids(sg_pic* h, int* n_grids, int* levels, int* coeffs, int cap) {
  SG_H(h);
  return h->e->get_grids(n_grids, levels, coeffs, cap);
}

int sg_pic_save(sg_pic* h, void* buf, size_t* size) {
  SG_H(h);
  if (!size) return invalid("sg_pic_save: size is NULL");
  return h->e->save(buf, size);
}

int sg_pic_load(sg_pic* h, const void* buf, size_t size) {
  SG_H(h);
  return h->e->load(buf, size);
}

int sg_pic_device_particles(sg_pic* h, sg_particles_out* out) {
  SG_H(h);
  if (!out) return invalid("sg_pic_device_particles: out is NULL");
  return h->e->device_particles(out);
}

int sg_pic_kernel_launches(sg_pic* h, unsigned long long* count) {
  SG_H(h);
  if (!count) return invalid("sg_pic_kernel_launches: count is NULL");
  *count = h->e->kernel_launches();
  return SG_OK;
}

int sg_pic_set_profiling(sg_pic* h, int on) {
  SG_H(h);
  return h->e->set_profiling(on);
}

int sg_pic_set_solve_variant(sg_pic* h, int variant) {
  SG_H(h);
  return h->e->set_solve_variant(variant);
}

int sg_pic_stage_times(sg_pic* h, double* ms, int cap) {
  SG_H(h);
  if (!ms) return invalid("sg_pic_stage_times: NULL buffer");
  return h->e->stage_times(ms, cap);
}

void sg_pic_destroy(sg_pic* h) {
  if (!h) return;
  delete h->e;
  delete h;
}

// ---------------------------------------------------------------- stand-alone sort
int sg_cell_sort(int precision, int dim, int level, size_t n, const void* const* u, uint32_t* keys_sorted,
                 uint32_t* perm, uint32_t* counts, void* stream) {
  if (dim != 2 && dim != 3) return invalid("sg_cell_sort: dim must be 2 or 3");
  if (level < 1 || dim * level > 24) return invalid("sg_cell_sort: need 1 <= level and dim*level <= 24");
  if (precision != SG_FP32 && precision != SG_FP64) return invalid("sg_cell_sort: bad precision");
  if (n > 0xFFFFFFF0ull) return invalid("sg_cell_sort: too many positions");
  if (n > 0 && (!u || !keys_sorted || !perm)) return invalid("sg_cell_sort: NULL pointer");
  for (int m = 0; n > 0 && m < dim; ++m)
    if (!u[m]) return invalid("sg_cell_sort: NULL position array");
  cudaStream_t s = (cudaStream_t)stream;
  size_t cells = (size_t)1 << (dim * level);
  if (n == 0) {
    if (counts) SG_CUDA(cudaMemsetAsync(counts, 0, cells * 4, s));
    return SG_OK;
  }
  size_t scr_words = sort_scratch_words(n);
  size_t words = 3 * n + scr_words + 4;
  uint32_t* buf = nullptr;
  SG_CUDA(cudaMallocAsync((void**)&buf, words * 4, s));
  uint32_t* keys = buf;
  uint32_t* vals = buf + n;
  uint32_t* keys_alt = buf + 2 * n;
  uint32_t* scr = buf + 3 * n;
  unsigned* status = (unsigned*)(scr + scr_words);
  SortScratch sc;
  sort_scratch_bind(sc, scr, n);
  int st = SG_OK;
  if (precision == SG_FP32) {
    st = dim == 2 ? launch_keys_raw<float, 2>((const float* const*)u, n, level, keys, nullptr, nullptr, status, s)
                  : launch_keys_raw<float, 3>((const float* const*)u, n, level, keys, nullptr, nullptr, status, s);
  } else {
    st = dim == 2 ? launch_keys_raw<double, 2>((const double* const*)u, n, level, keys, nullptr, nullptr, status, s)
                  : launch_keys_raw<double, 3>((const double* const*)u, n, level, keys, nullptr, nullptr, status, s);
  }
  bool in_alt = false;
  // the sorted result lands in (keys, vals) or (keys_alt, perm) depending on the pass count
  if (st == SG_OK) st = radix_sort_pairs(keys, vals, keys_alt, perm, n, dim * level, true, sc, s, &in_alt);
  if (st == SG_OK) {
    const uint32_t* ks = in_alt ? keys_alt : keys;
    const uint32_t* ps = in_alt ? perm : vals;
    if (ks != keys_sorted) {
      cudaError_t e = cudaMemcpyAsync(keys_sorted, ks, n * 4, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) st = SG_ERR_CUDA;
    }
    if (st == SG_OK && ps != perm) {
      cudaError_t e = cudaMemcpyAsync(perm, ps, n * 4, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) st = SG_ERR_CUDA;
    }
    if (st == SG_OK && counts) {
      cudaError_t e = cudaMemsetAsync(counts, 0, cells * 4, s);
      if (e != cudaSuccess) st = SG_ERR_CUDA;
      if (st == SG_OK) st = launch_counts(keys_sorted, n, counts, s);
    }
  }
  cudaFreeAsync(buf, s);
  return st;
}

}  // extern "C"
