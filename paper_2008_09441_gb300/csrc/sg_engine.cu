// Engine<real, D>: one sparse-grid PIC run on one GPU, the host runtime
// around the kernels:
// - device buffers from the stream-ordered allocator (freed memory stays in
//   the pool for the next run);
// - the step as CUDA graphs, one per (particle buffer, sort or not); a sort
//   step's counting sort runs on a second stream beside the grid stages;
// - the step split for the cross-run solve of batched serving, and for
//   sharded runs around the exchange of the regular-grid density;
// - the init-time autotuner (solve variant, push grid, deposit window) with
//   a process-wide cache per run shape;
// - FP64 diagnostics written by one kernel into mapped pinned records,
//   blocking or pipelined.
#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "sg_engine.cuh"

namespace sg {

// Sort period when the caller passes 0.  The step sort restores the deposit
// window's locality at the price of one payload scatter.  Measured mean
// steps: on the 2D n = 10 Landau workload (4.2 M particles, about 4 cells of
// drift per step) a sort every 4 steps is shortest; on the 3D n = 7
// two-stream workload (16.8 M particles, whose sort moves 28 B each) every 6.
constexpr int default_sort_every(int dim) { return dim == 3 ? 6 : 4; }

std::vector<GridSpec> combination_grids(int d, int n, int tau) {
  std::vector<GridSpec> out;
  for (int q = 0; q < d; ++q) {
    int target = n + (d - 1) * tau - q;
    int binom = (d == 3 && q == 1) ? 2 : 1;  // C(d-1, q) for d <= 3
    int coeff = (q % 2 ? -1 : 1) * binom;
    if (d == 2) {
      for (int a = tau; a <= n; ++a)
        for (int b = tau; b <= n; ++b)
          if (a + b == target) out.push_back({{a, b, 0}, coeff});
    } else {
      for (int a = tau; a <= n; ++a)
        for (int b = tau; b <= n; ++b)
          for (int c = tau; c <= n; ++c)
            if (a + b + c == target) out.push_back({{a, b, c}, coeff});
    }
  }
  return out;
}

namespace {

// Process-wide record of the solve-variant timings, by grid set.
struct TuneKey {
  int real_bytes, dim, n, tau;
  bool operator<(const TuneKey& o) const {
    return std::tie(real_bytes, dim, n, tau) < std::tie(o.real_bytes, o.dim, o.n, o.tau);
  }
};
struct TuneEntry {
  int mode;
  float ms[2];
};
std::map<TuneKey, TuneEntry>& tune_cache() {
  static std::map<TuneKey, TuneEntry> m;
  return m;
}
std::mutex& tune_mu() {
  static std::mutex m;
  return m;
}

// Process-wide record of the particle-pass tuner, by the run's shape: the
// precision, dimension, level, particle count (log2 bucket), centring and
// push kind.
constexpr int kPushCands = 3;   // push grids: half, one and two resident waves
constexpr int kDepCands = 4;    // deposit window capacities (64-bit-equivalent nodes)
constexpr int kDepCap[kDepCands] = {4096, 6144, 8192, 12288};
struct PartKey {
  int real_bytes, dim, n, np_log2, cell, boris;
  bool operator<(const PartKey& o) const {
    return std::tie(real_bytes, dim, n, np_log2, cell, boris) <
           std::tie(o.real_bytes, o.dim, o.n, o.np_log2, o.cell, o.boris);
  }
};
struct PartEntry {
  int push_pick, dep_pick;
  float push_ms[kPushCands], dep_ms[kDepCands];
  bool refined;                  // the window was re-chosen on drifted particles
  float dep_drift_ms[kDepCands];  // the deposit timed before the first sort step
};
std::map<PartKey, PartEntry>& part_cache() {
  static std::map<PartKey, PartEntry> m;
  return m;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

template <typename real, int D>
class Engine final : public EngineBase {
 public:
  ~Engine() override { release(); }

  int init(const EngineConfig& cfg, const sg_particles* parts, cudaStream_t stream) override {
    cfg_ = cfg;
    n_ = cfg.n;
    N_ = 1 << n_;
    ND_ = (size_t)1;
    for (int m = 0; m < D; ++m) ND_ *= (size_t)N_;
    np_ = parts->n;
    if (stream) {
      stream_ = stream;
      own_stream_ = false;
    } else {
      SG_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
      own_stream_ = true;
    }
    SG_CUDA(cudaStreamCreateWithFlags(&sort_stream_, cudaStreamNonBlocking));
    SG_CUDA(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
    SG_CUDA(cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming));
    sort_every_ = cfg.sort_every > 0 ? cfg.sort_every : default_sort_every(D);
    tau_ = cfg.tau == SG_TAU_ADAPTIVE ? 1 : cfg.tau;
    adaptive_ = cfg.tau == SG_TAU_ADAPTIVE;

    // ---- particles (two sets for the sort's out-of-place permutation)
    size_t pb = std::max<size_t>(np_, 1);
    for (int set = 0; set < 2; ++set) {
      for (int m = 0; m < D; ++m) {
        SG_TRY(alloc((void**)&P_[set].u[m], pb * sizeof(real)));
        SG_TRY(alloc((void**)&P_[set].v[m], pb * sizeof(real)));
      }
      SG_TRY(alloc((void**)&P_[set].w, pb * sizeof(real)));
      SG_TRY(alloc((void**)&P_[set].pid, pb * sizeof(uint32_t)));
    }
    // ---- small device records (the status word is written by the upload check)
    SG_TRY(alloc((void**)&dd_, sizeof(DevDiag)));
    SG_TRY(alloc((void**)&status_, sizeof(unsigned)));
    SG_TRY(alloc((void**)&checksum_, sizeof(unsigned long long)));
    SG_CUDA(cudaMemsetAsync(dd_, 0, sizeof(DevDiag), stream_));
    SG_CUDA(cudaMemsetAsync(status_, 0, sizeof(unsigned), stream_));
    SG_CUDA(cudaMemsetAsync(checksum_, 0, sizeof(unsigned long long), stream_));

    cur_ = 0;
    SG_TRY(upload_particles(parts));
    SG_TRY(alloc((void**)&keys_, pb * 4));
    SG_TRY(alloc((void**)&keys_alt_, pb * 4));
    tile_shift_ = std::max(0, n_ - 12 / D);
    ntiles_ = (size_t)1 << (D * (n_ - tile_shift_));
    SG_TRY(alloc((void**)&tile_count_, ntiles_ * 4));
    SG_TRY(alloc((void**)&cursor_, ntiles_ * 4));
    SG_TRY(alloc((void**)&scan_sums_, scan_block_sums_words(ntiles_) * 4));
    // push grid: one resident wave by default; the tuner may take half or two
    // waves, so the kinetic-energy partials (one per block) fit two waves
    push_wave_ = push_blocks<real, D>(np_);
    push_blocks_ = push_wave_;
    nke_ = push_blocks_;
    win_cap_ = cfg_.win_cap;
    SG_TRY(alloc((void**)&ke_partials_, (size_t)2 * push_wave_ * sizeof(double)));
    SG_CUDA(cudaMemsetAsync(ke_partials_, 0, (size_t)2 * push_wave_ * sizeof(double), stream_));

    // ---- regular grid, combined field, twiddles
    SG_TRY(alloc((void**)&rho_reg_, ND_ * sizeof(real)));
    SG_TRY(alloc((void**)&Ehi_, (size_t)ec_stride<D>() * ND_ * sizeof(real)));  // node-interleaved
    if (sizeof(real) == 4) SG_TRY(alloc((void**)&Elo_, (size_t)D * ND_ * sizeof(float)));
    nrows_ = (int)(ND_ / (size_t)N_);
    SG_TRY(alloc((void**)&fe_partials_, (size_t)nrows_ * D * sizeof(double)));  // per (line, component)
    SG_TRY(alloc((void**)&comb_counter_, sizeof(unsigned)));
    SG_CUDA(cudaMemsetAsync(comb_counter_, 0, sizeof(unsigned), stream_));
    {
      const std::vector<cplx<real>> tw = make_twiddles<real>(n_);
      SG_TRY(alloc((void**)&tw_, tw.size() * sizeof(cplx<real>)));
      // pageable source: staged when the call returns, no synchronisation needed
      SG_CUDA(cudaMemcpyAsync(tw_, tw.data(), tw.size() * sizeof(cplx<real>), cudaMemcpyHostToDevice, stream_));
    }
    filter_ = cfg.mode == SG_MODE_FILTER;
    if (filter_) {
      SG_TRY(alloc((void**)&rho_f_, ND_ * sizeof(real)));
      SG_TRY(alloc((void**)&regA_, ND_ * sizeof(cplx<real>)));
      SG_TRY(alloc((void**)&regB_, ND_ * sizeof(cplx<real>)));
      std::vector<real> kt((size_t)D * N_);
      for (int m = 0; m < D; ++m)
        for (int i = 0; i < N_; ++i)
          kt[(size_t)m * N_ + i] = (real)(2.0 * M_PI / cfg_.L[m] * (double)(i < N_ / 2 ? i : i - N_));
      SG_TRY(alloc((void**)&ktab_, kt.size() * sizeof(real)));
      SG_CUDA(cudaMemcpyAsync(ktab_, kt.data(), kt.size() * sizeof(real), cudaMemcpyHostToDevice, stream_));
      reg_blocks_ = (int)std::min<size_t>(152 * 8, (ND_ + 255) / 256);
      SG_TRY(alloc((void**)&reg_partials_, (size_t)2 * reg_blocks_ * sizeof(double)));
    }

    SG_TRY(particle_stats());

    SG_TRY(build_grid_set(tau_));
    // Initial state: sort, fields at t = 0, backward half kick.
    SG_TRY(enqueue_sort());
    if (cfg.deferred) {  // the caller sums the density across the run's parts, then start()
      if (adaptive_) {
        set_error("sg_pic_init_deferred: adaptive tau needs the whole run's particle count (not supported)");
        return SG_ERR_UNSUPPORTED;
      }
      SG_TRY(enqueue_deposit());
      SG_CUDA(cudaStreamSynchronize(stream_));
      phase_ = kAwaitStart;
      step_ = 0;
      return check_status();
    }
    if (adaptive_) {  // Algorithm 1 on the initial density picks the first tau
      SG_TRY(enqueue_deposit());
      int t = tau_;
      const int st = select_tau(&t, nullptr, nullptr, 0);
      if (st == SG_OK && t != tau_) {
        SG_CUDA(cudaStreamSynchronize(stream_));
        SG_TRY(build_grid_set(t));
      } else if (st != SG_OK && st != SG_ERR_RANGE) {
        return st;
      }
      SG_TRY(enqueue_restrict_solve_combine());
    } else {
      SG_TRY(enqueue_fields());
    }
    if (!filter_) {  // pick the solve variant, then recompute with it
      SG_TRY(tune_solve());
      SG_TRY(enqueue_combine(false));
    }
    SG_TRY(tune_particles());
    SG_TRY(enqueue_push(-0.5 * cfg_.dt, false, nullptr));
    SG_CUDA(cudaStreamSynchronize(stream_));
    step_ = 0;
    return check_status();
  }

  // The uploaded particles' statistics, one pass and one synchronisation
  // (the kernel writes into mapped pinned memory): sum_p q_p in FP64 (fixed
  // while the particles are), max_p |q_p| for the deposit's fixed-point
  // scale, and the status word of the upload's finiteness check.
  int particle_stats() {
    const int nb = 256;
    SG_TRY(ensure_pinned(&stats_host_, &stats_host_bytes_, (2 * nb + 1) * sizeof(double)));
    double* h = static_cast<double*>(stats_host_);
    void* hd = nullptr;
    SG_CUDA(cudaHostGetDevicePointer(&hd, stats_host_, 0));
    if (np_ > 0) {
      SG_TRY(launch_charge_stats<real>(P_[cur_].w, np_, status_, static_cast<double*>(hd), nb, stream_));
      SG_CUDA(cudaStreamSynchronize(stream_));
    } else {
      std::memset(h, 0, (2 * nb + 1) * sizeof(double));
    }
    charge_total_ = 0;
    double qmax = 0;
    for (int b = 0; b < nb; ++b) {
      charge_total_ += h[b];
      qmax = std::max(qmax, h[nb + b]);
    }
    unsigned long long stw = 0;
    std::memcpy(&stw, h + 2 * nb, sizeof(stw));
    if ((unsigned)stw & ST_NONFINITE) {
      set_error("non-finite particle position, velocity or charge");
      return SG_ERR_NONFINITE;
    }
    set_deposit_scale(qmax);
    return SG_OK;
  }

  // Sharded runs.  start(): the fields of the (summed) regular-grid density
  // and the backward half kick, completing a deferred init.  step_deposit /
  // step_fields: the two halves of sg_pic_step around the exchange of the
  // density (push, sort when due and deposit; restriction, solves,
  // combination), direct launches.
  int start() override {
    if (phase_ != kAwaitStart) {
      set_error("sg_pic_start: the run was not created by sg_pic_init_deferred, or has started");
      return SG_ERR_STATE;
    }
    SG_TRY(enqueue_restrict_solve_combine());
    if (!filter_) {
      SG_TRY(tune_solve());
      SG_TRY(enqueue_combine(false));
    }
    SG_TRY(enqueue_push(-0.5 * cfg_.dt, false, nullptr));
    SG_CUDA(cudaStreamSynchronize(stream_));
    phase_ = kReady;
    return check_status();
  }
  int step_deposit() override {
    if (phase_ != kReady || adaptive_) {
      set_error(adaptive_ ? "sg_pic_step_deposit: not supported with adaptive tau"
                          : "sg_pic_step_deposit: the run is not between steps");
      return adaptive_ ? SG_ERR_UNSUPPORTED : SG_ERR_STATE;
    }
    const bool do_sort = ((step_ + 1) % sort_every_) == 0;
    const unsigned long long l0 = launches_so_far();
    SG_TRY(enqueue_push(cfg_.dt, true, ke_partials_, do_sort));
    if (do_sort) SG_TRY(sort_finish());
    SG_TRY(enqueue_deposit());
    launches_ += launches_so_far() - l0;
    phase_ = kHalfStep;
    return SG_OK;
  }
  int step_fields() override {
    if (phase_ != kHalfStep) {
      set_error("sg_pic_step_fields: sg_pic_step_deposit must come first");
      return SG_ERR_STATE;
    }
    const unsigned long long l0 = launches_so_far();
    SG_TRY(enqueue_restrict_solve_combine(ke_partials_));
    launches_ += launches_so_far() - l0;
    ++step_;
    phase_ = kReady;
    return SG_OK;
  }
  int set_charge_total(double q) override {
    if (!std::isfinite(q)) {
      set_error("sg_pic_set_charge_total: non-finite charge");
      return SG_ERR_INVALID;
    }
    charge_total_ = q;
    invalidate_graphs();  // the restriction's mean is a launch argument
    return SG_OK;
  }
  int density_copy(void* dev_buf, size_t n, int to_run) override {
    if (!dev_buf) {
      set_error("sg_pic_density_copy: NULL buffer");
      return SG_ERR_INVALID;
    }
    if (n != ND_) return size_error("sg_pic_density_copy");
    if (to_run)
      SG_CUDA(cudaMemcpyAsync(rho_reg_, dev_buf, ND_ * sizeof(real), cudaMemcpyDeviceToDevice, stream_));
    else
      SG_CUDA(cudaMemcpyAsync(dev_buf, rho_reg_, ND_ * sizeof(real), cudaMemcpyDeviceToDevice, stream_));
    SG_CUDA(cudaStreamSynchronize(stream_));
    return SG_OK;
  }

  int step(int nsteps) override {
    if (nsteps < 0) {
      set_error("sg_pic_step: nsteps < 0");
      return SG_ERR_INVALID;
    }
    if (phase_ != kReady) {
      set_error(phase_ == kAwaitStart ? "sg_pic_step: a deferred run needs sg_pic_start first"
                                      : "sg_pic_step: finish the split step with sg_pic_step_fields first");
      return SG_ERR_STATE;
    }
    if (profiling_) std::fill(stage_ms_, stage_ms_ + 6, 0.0);
    for (int k = 0; k < nsteps; ++k) {
      bool do_sort = ((step_ + 1) % sort_every_) == 0;
      if (adaptive_) {
        SG_TRY(step_adaptive(do_sort));
      } else if (profiling_) {
        SG_TRY(step_profiled(do_sort));
      } else {
        if (do_sort && refine_pending_) SG_TRY(refine_deposit());
        SG_TRY(step_graph(do_sort));
      }
      ++step_;
    }
    return SG_OK;
  }

  // Diagnostics read-back in pinned memory: the device record, the count
  // checksum, the status word, then one FP64 charge per component grid.
  static size_t diag_off_cks() { return (sizeof(DevDiag) + 15) / 16 * 16; }
  size_t diag_bytes() const { return diag_off_cks() + 16 + (size_t)ngrids_ * sizeof(double); }

  // Host-side state a record is read against, taken when its copies are
  // enqueued (the grid set may change before the record is read).
  struct DiagMeta {
    long long step = 0;
    int tau = 0;
    double charge_total = 0;
    double mean_charge = 0;  // the charge of the mean density the grids are stored without
    std::vector<double> coeff;
  };
  DiagMeta diag_meta() const {
    DiagMeta m;
    m.step = step_;
    m.tau = tau_;
    m.charge_total = charge_total_;
    m.mean_charge = (double)rho_mean() * box_volume();
    m.coeff.resize(ngrids_);
    for (int i = 0; i < ngrids_; ++i) m.coeff[i] = (double)grids_[i].coeff;
    return m;
  }
  // Pinned host memory mapped into the device's address space: the record
  // kernel writes a diagnostics record straight into it.
  int ensure_pinned(void** p, size_t* have, size_t need) {
    if (need <= *have) return SG_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *have = 0;
    SG_CUDA(cudaHostAlloc(p, need, cudaHostAllocMapped));
    *have = need;
    return SG_OK;
  }
  // Enqueue the kernel that packs the record into the mapped host buffer h
  // (no copy operation on the stream: a copy after every step cost about
  // 17 us of stream time between the step's kernels and the next step's).
  int enqueue_diag(char* h) {
    const size_t o_cks = diag_off_cks(), o_ch = o_cks + 16;
    void* hd = nullptr;
    SG_CUDA(cudaHostGetDevicePointer(&hd, h, 0));
    return launch_diag_record<real>(grids_dev_, ngrids_, rho_arena_, dd_, checksum_, status_, hd, o_cks, o_ch,
                                    stream_);
  }
  // Convert a landed record (FP64 charge sums over the grids on the host).
  int read_diag(const char* h, const DiagMeta& m, sg_diag* out) {
    const size_t o_cks = diag_off_cks(), o_st = o_cks + 8, o_ch = o_cks + 16;
    const int ng = (int)m.coeff.size();
    DevDiag dd;
    std::memcpy(&dd, h, sizeof(DevDiag));
    unsigned long long cks = 0;
    std::memcpy(&cks, h + o_cks, 8);
    unsigned st = 0;
    std::memcpy(&st, h + o_st, sizeof(unsigned));
    std::memset(out, 0, sizeof(*out));
    out->step = m.step;
    out->t = (double)m.step * cfg_.dt;
    out->tau = m.tau;
    out->n_grids = ng;
    out->charge_total = m.charge_total;
    double comb = 0, maxerr = 0;
    for (int i = 0; i < ng; ++i) {
      double ch;
      std::memcpy(&ch, h + o_ch + (size_t)i * sizeof(double), sizeof(double));
      ch += m.mean_charge;
      comb += m.coeff[i] * ch;
      maxerr = std::max(maxerr, std::fabs(ch - m.charge_total));
    }
    out->charge_combined = comb;
    out->charge_grid_max_abs_err = maxerr;
    out->field_energy = dd.field_energy;
    out->field_energy_prev = dd.field_energy_prev;
    out->kinetic_energy = dd.kinetic_energy;
    out->count_checksum = cks;
    if (st & ST_NONFINITE) {
      set_error("a kernel produced a non-finite particle state");
      return SG_ERR_NONFINITE;
    }
    return SG_OK;
  }

  int diagnostics(sg_diag* out) override {
    // one synchronisation for the whole record
    SG_TRY(ensure_pinned(&diag_host_, &diag_host_bytes_, diag_bytes()));
    char* h = static_cast<char*>(diag_host_);
    SG_TRY(enqueue_diag(h));
    SG_CUDA(cudaStreamSynchronize(stream_));
    return read_diag(h, diag_meta(), out);
  }

  // Pipelined diagnostics: records enqueued into a ring of pinned slots and
  // read in order, so that a monitor reads step k while step k+1 runs.
  int diagnostics_post() override {
    if (ring_count_ == kDiagRing) {
      set_error("sg_pic_diagnostics_post: every slot holds a record not yet collected");
      return SG_ERR_STATE;
    }
    DiagSlot& s = ring_[(ring_head_ + ring_count_) % kDiagRing];
    SG_TRY(ensure_pinned(&s.host, &s.bytes, diag_bytes()));
    if (!s.ev) SG_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
    SG_TRY(enqueue_diag(static_cast<char*>(s.host)));
    SG_CUDA(cudaEventRecord(s.ev, stream_));
    s.meta = diag_meta();
    ++ring_count_;
    return SG_OK;
  }
  int diagnostics_collect(sg_diag* out) override {
    if (ring_count_ == 0) {
      set_error("sg_pic_diagnostics_collect: no record was posted");
      return SG_ERR_STATE;
    }
    DiagSlot& s = ring_[ring_head_];
    ring_head_ = (ring_head_ + 1) % kDiagRing;
    --ring_count_;
    SG_CUDA(cudaEventSynchronize(s.ev));
    return read_diag(static_cast<const char*>(s.host), s.meta, out);
  }

  int select_tau(int* tau, double* est_grid, double* est_noise, int cap) override {
    int hi = D == 2 ? n_ - 3 : n_ - 2;
    if (hi < 1) {
      set_error("sg_pic_select_tau: empty tau range [1, n-3] (2D) / [1, n-2] (3D)");
      return SG_ERR_RANGE;
    }
    for (int m = 1; m < D; ++m)
      if (std::fabs(cfg_.L[m] - cfg_.L[0]) > 1e-12 * std::fabs(cfg_.L[0])) {
        set_error("sg_pic_select_tau: the estimates assume a cubic box (one L)");
        return SG_ERR_UNSUPPORTED;
      }
    SG_TRY(ensure_estimator_buffers());
    const double L = cfg_.L[0];
    // rho~ of the current positions (the deposit of the last step).
    SG_TRY(launch_to_double<real>(rho_reg_, est_rho_, ND_, stream_));
    SG_TRY(launch_real_to_cplx(est_rho_, est_z_, ND_, 1.0 / (double)ND_, stream_));
    for (int ax = 0; ax < D; ++ax) SG_TRY(launch_fft_array_axis<double>(est_z_, D, n_, ax, false, tw64_, n_, stream_));
    SG_TRY(launch_maxabs_cplx(est_z_, ND_, est_scalar_ + 0, stream_));
    const double Pc = (double)np_ / (double)ND_;
    const double frac = cfg_.alpha * std::sqrt(cfg_.pc_ref / Pc);
    SG_TRY(launch_threshold(est_z_, ND_, est_scalar_ + 0, frac, stream_));
    double kfac[3] = {0, 0, 0};
    for (int m = 0; m < D; ++m) kfac[m] = 2.0 * M_PI / cfg_.L[m];
    // masks: kappa_m (single axis), beta (pairs), gamma (all three)
    std::vector<int> masks;
    for (int m = 0; m < D; ++m) masks.push_back(1 << m);
    if (D == 2) {
      masks.push_back(3);
    } else {
      masks.push_back(3);  // xy
      masks.push_back(6);  // yz
      masks.push_back(5);  // zx
      masks.push_back(7);  // xyz
    }
    const bool paper = cfg_.tau_constants == SG_TAU_CONST_PAPER;
    for (size_t i = 0; i < masks.size(); ++i) {
      if (paper) {
        SG_TRY(launch_kmult(est_z_, est_w_, D, n_, kfac, masks[i], stream_));
        for (int ax = 0; ax < D; ++ax)
          SG_TRY(launch_fft_array_axis<double>(est_w_, D, n_, ax, true, tw64_, n_, stream_));
        SG_TRY(launch_maxabs_real_part(est_w_, ND_, est_scalar_ + 1 + i, stream_));
      } else {
        SG_TRY(launch_maxabs_kmult(est_z_, D, n_, kfac, masks[i], est_scalar_ + 1 + i, stream_));
      }
    }
    SG_TRY(launch_maxabs_real(est_rho_, ND_, est_scalar_ + 8, stream_));
    double sc[9];
    SG_CUDA(cudaMemcpyAsync(sc, est_scalar_, sizeof(sc), cudaMemcpyDeviceToHost, stream_));
    SG_CUDA(cudaStreamSynchronize(stream_));
    double kappa[3] = {0, 0, 0}, beta[3] = {0, 0, 0}, gamma = 0, sigma;
    const double Q = std::fabs(charge_total_);
    if (paper) {
      for (int m = 0; m < D; ++m) kappa[m] = 0.25 * sc[1 + m];
      if (D == 2) {
        beta[0] = sc[1 + 2] / 72.0;
      } else {
        beta[0] = sc[1 + 3] / 72.0;
        beta[1] = sc[1 + 4] / 72.0;
        beta[2] = sc[1 + 5] / 72.0;
        gamma = sc[1 + 6] / 864.0;
      }
      sigma = std::sqrt(std::pow(2.0 / 3.0, D) * Q * sc[8]);
    } else {
      for (int m = 0; m < D; ++m) kappa[m] = sc[1 + m];
      if (D == 2) {
        beta[0] = sc[1 + 2];
      } else {
        beta[0] = sc[1 + 3];
        beta[1] = sc[1 + 4];
        beta[2] = sc[1 + 5];
        gamma = sc[1 + 6];
      }
      sigma = std::sqrt(Q * sc[8]);
    }
    const double h = L / (double)N_;
    int best = 1;
    double best_total = 0;
    for (int t = 1; t <= hi; ++t) {
      const double m = (double)(n_ - t);
      double g, z;
      if (D == 2) {
        g = h * h * (kappa[0] + kappa[1] + beta[0] * L * L * std::pow(2.0, -2.0 * t) * (5 * m + 1));
        z = sigma * std::pow(2.0, 0.5 * (t - 1)) * (m * (1 + std::sqrt(2.0)) + std::sqrt(2.0)) /
            std::sqrt((double)np_ * h * L);
      } else {
        g = h * h *
            (kappa[0] + kappa[1] + kappa[2] + (beta[0] + beta[1] + beta[2]) * L * L * std::pow(2.0, -2.0 * t) * (5 * m + 1) +
             gamma * std::pow(L, 4) * std::pow(2.0, -(4.0 * t + 1)) * (25 * m * m - 5 * m + 2));
        z = sigma * std::pow(2.0, (double)(t - 2)) *
            ((3 + std::sqrt(2.0)) * m * m + (5 + std::sqrt(2.0)) * m + 4) / std::sqrt((double)np_ * h * L * L);
      }
      if (est_grid && t <= cap) est_grid[t - 1] = g;
      if (est_noise && t <= cap) est_noise[t - 1] = z;
      if (t == 1 || g + z < best_total) {
        best = t;
        best_total = g + z;
      }
    }
    *tau = best;
    return SG_OK;
  }

  int set_tau(int tau) override {
    if (tau < 1 || tau > n_) {
      set_error("sg_pic_set_tau: tau outside [1, n]");
      return SG_ERR_INVALID;
    }
    if (tau == tau_) return SG_OK;
    SG_CUDA(cudaStreamSynchronize(stream_));
    SG_TRY(build_grid_set(tau));
    SG_TRY(enqueue_restrict());
    if (filter_) return enqueue_filter_field(nullptr);
    SG_TRY(tune_solve());
    SG_TRY(enqueue_combine(true, nullptr));
    return SG_OK;
  }

  int get_particles(const sg_particles_out* out) override {
    if (!out || out->n != np_) {
      set_error("sg_pic_get_particles: out->n must equal the run's particle count");
      return SG_ERR_SIZE;
    }
    if (np_ == 0) return SG_OK;
    PArrays<real, D> dst;
    std::vector<void*> temps;
    for (int m = 0; m < D; ++m) {
      dst.u[m] = (real*)out->u[m];
      dst.v[m] = (real*)out->v[m];
    }
    dst.w = (real*)out->w;
    dst.pid = nullptr;
    if (!out->on_device) {
      // stage in the other particle set (free between steps)
      const int o = cur_ ^ 1;
      for (int m = 0; m < D; ++m) {
        dst.u[m] = P_[o].u[m];
        dst.v[m] = P_[o].v[m];
      }
      dst.w = P_[o].w;
    }
    SG_TRY(launch_unpermute<real, D>(P_[cur_], dst, np_, stream_));
    if (!out->on_device) {
      for (int m = 0; m < D; ++m) {
        if (out->u[m]) SG_CUDA(cudaMemcpyAsync(out->u[m], dst.u[m], np_ * sizeof(real), cudaMemcpyDeviceToHost, stream_));
        if (out->v[m]) SG_CUDA(cudaMemcpyAsync(out->v[m], dst.v[m], np_ * sizeof(real), cudaMemcpyDeviceToHost, stream_));
      }
      if (out->w) SG_CUDA(cudaMemcpyAsync(out->w, dst.w, np_ * sizeof(real), cudaMemcpyDeviceToHost, stream_));
    }
    SG_CUDA(cudaStreamSynchronize(stream_));
    return SG_OK;
  }

  int get_keys(uint32_t* keys, uint32_t* counts, size_t cap_keys, size_t cap_counts) override {
    if (keys && cap_keys < np_) {
      set_error("sg_pic_get_keys: key buffer too small");
      return SG_ERR_SIZE;
    }
    if (counts && cap_counts < ND_) {
      set_error("sg_pic_get_keys: count buffer too small");
      return SG_ERR_SIZE;
    }
    SG_TRY(launch_keys<real, D>(P_[cur_], np_, n_, keys_alt_, nullptr, nullptr, status_, stream_));
    if (keys) SG_CUDA(cudaMemcpyAsync(keys, keys_alt_, np_ * 4, cudaMemcpyDeviceToHost, stream_));
    if (counts) {
      uint32_t* dcounts = nullptr;
      SG_TRY(alloc((void**)&dcounts, ND_ * 4));
      SG_CUDA(cudaMemsetAsync(dcounts, 0, ND_ * 4, stream_));
      SG_TRY(launch_counts(keys_alt_, np_, dcounts, stream_));
      SG_CUDA(cudaMemcpyAsync(counts, dcounts, ND_ * 4, cudaMemcpyDeviceToHost, stream_));
      SG_CUDA(cudaStreamSynchronize(stream_));
      free_one(dcounts);
    }
    SG_CUDA(cudaStreamSynchronize(stream_));
    return SG_OK;
  }

  int get_field(double* E, size_t cap) override {
    if (cap < (size_t)D * ND_) return size_error("sg_pic_get_field");
    double* tmp = nullptr;
    SG_TRY(alloc((void**)&tmp, (size_t)D * ND_ * sizeof(double)));
    SG_TRY(launch_field_to_double<real>(Ehi_, Elo_, tmp, ND_, D, ec_stride<D>(), stream_));
    SG_CUDA(cudaMemcpyAsync(E, tmp, (size_t)D * ND_ * sizeof(double), cudaMemcpyDeviceToHost, stream_));
    SG_CUDA(cudaStreamSynchronize(stream_));
    free_one(tmp);
    return SG_OK;
  }

  int get_grid_charge(double* rho, size_t cap) override {
    if (cap < S_) return size_error("sg_pic_get_grid_charge");
    SG_TRY(copy_to_host_double(rho_arena_, rho, S_));
    return add_mean(rho, S_);
  }

  int get_grid_field(double* E, size_t cap) override {
    if (filter_) {
      set_error("sg_pic_get_grid_field: the filter mode solves no component fields");
      return SG_ERR_STATE;
    }
    if (cap < (size_t)D * S_) return size_error("sg_pic_get_grid_field");
    std::vector<double> all((size_t)D * S_);
    SG_TRY(copy_to_host_double(E_arena_, all.data(), (size_t)D * S_));
    size_t o = 0;
    for (int g = 0; g < ngrids_; ++g) {
      size_t sz = (size_t)gdesc_[g].size, off = (size_t)gdesc_[g].offset;
      for (int m = 0; m < D; ++m) {
        std::memcpy(E + o, all.data() + (size_t)m * S_ + off, sz * sizeof(double));
        o += sz;
      }
    }
    return SG_OK;
  }

  int get_regular_charge(double* rho, size_t cap) override {
    if (cap < ND_) return size_error("sg_pic_get_regular_charge");
    return copy_to_host_double(rho_reg_, rho, ND_);
  }

  // The density the field comes from, on the regular nodes: the combination
  // sum_i c_i P_i rho_i of the component densities (eq. sparse_filter; in
  // the filter mode the density its regular-grid solve used).
  int get_density(double* rho, size_t cap) override {
    if (cap < ND_) return size_error("sg_pic_get_density");
    if (filter_) {
      SG_TRY(copy_to_host_double(rho_f_, rho, ND_));
      return add_mean(rho, ND_);
    }
    real* tmp = nullptr;
    SG_TRY(alloc((void**)&tmp, ND_ * sizeof(real)));
    CombineFinal off;
    std::memset(&off, 0, sizeof(off));
    int st = launch_combine<real, D>(grids_dev_, levels_, lmin_, rho_arena_, S_, n_, tmp, nullptr, fe_partials_, off,
                                     stream_, 1, cfg_.cell, cfg_.combine_fp64);
    if (st == SG_OK) st = copy_to_host_double(tmp, rho, ND_);
    free_one(tmp);
    if (st == SG_OK) add_mean(rho, ND_);
    return st;
  }

  int get_grids(int* n_grids, int* levels, int* coeffs, int cap) override {
    if (n_grids) *n_grids = ngrids_;
    for (int g = 0; g < ngrids_ && g < cap; ++g) {
      if (levels)
        for (int m = 0; m < 3; ++m) levels[3 * g + m] = grids_[g].l[m];
      if (coeffs) coeffs[g] = grids_[g].coeff;
    }
    return SG_OK;
  }

  // Checkpoint layout: header, then u[d], v[d], w arrays in original order.
  struct Header {
    char magic[8];
    int version, dim, precision, n, tau, adaptive, mode, centring;
    long long np, step;
    double dt;
    DevDiag dd;
  };

  int save(void* buf, size_t* size) override {
    size_t need = sizeof(Header) + (size_t)(2 * D + 1) * np_ * sizeof(real);
    if (!buf || *size < need) {
      *size = need;
      return buf ? SG_ERR_SIZE : SG_OK;
    }
    Header hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "SGPICv2", 8);
    hd.version = 2;
    hd.mode = cfg_.mode;
    hd.centring = cfg_.cell ? SG_CELL_CENTRED : SG_NODE_CENTRED;
    hd.dim = D;
    hd.precision = sizeof(real) == 4 ? SG_FP32 : SG_FP64;
    hd.n = n_;
    hd.tau = tau_;
    hd.adaptive = adaptive_ ? 1 : 0;
    hd.np = (long long)np_;
    hd.step = step_;
    hd.dt = cfg_.dt;
    SG_CUDA(cudaMemcpyAsync(&hd.dd, dd_, sizeof(DevDiag), cudaMemcpyDeviceToHost, stream_));
    SG_CUDA(cudaStreamSynchronize(stream_));
    std::memcpy(buf, &hd, sizeof(hd));
    char* p = (char*)buf + sizeof(hd);
    sg_particles_out o;
    std::memset(&o, 0, sizeof(o));
    o.n = np_;
    o.on_device = 0;
    for (int m = 0; m < D; ++m) {
      o.u[m] = p + (size_t)m * np_ * sizeof(real);
      o.v[m] = p + (size_t)(D + m) * np_ * sizeof(real);
    }
    o.w = p + (size_t)(2 * D) * np_ * sizeof(real);
    SG_TRY(get_particles(&o));
    *size = need;
    return SG_OK;
  }

  int load(const void* buf, size_t size) override {
    if (!buf || size < sizeof(Header)) return size_error("sg_pic_load");
    Header hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "SGPICv2", 8) != 0 || hd.dim != D ||
        hd.precision != (sizeof(real) == 4 ? SG_FP32 : SG_FP64) || hd.n != n_ || hd.np != (long long)np_ ||
        hd.mode != cfg_.mode || hd.centring != (cfg_.cell ? SG_CELL_CENTRED : SG_NODE_CENTRED)) {
      set_error("sg_pic_load: checkpoint does not match this run (magic, dim, precision, level, particle count, "
                "mode or centring)");
      return SG_ERR_INVALID;
    }
    size_t need = sizeof(Header) + (size_t)(2 * D + 1) * np_ * sizeof(real);
    if (size < need) return size_error("sg_pic_load");
    const char* p = (const char*)buf + sizeof(hd);
    sg_particles in;
    std::memset(&in, 0, sizeof(in));
    in.n = np_;
    in.on_device = 0;
    for (int m = 0; m < D; ++m) {
      in.u[m] = p + (size_t)m * np_ * sizeof(real);
      in.v[m] = p + (size_t)(D + m) * np_ * sizeof(real);
    }
    in.w = p + (size_t)(2 * D) * np_ * sizeof(real);
    SG_CUDA(cudaStreamSynchronize(stream_));
    cur_ = 0;
    SG_TRY(upload_particles(&in));
    SG_TRY(particle_stats());
    if (hd.tau != tau_) SG_TRY(build_grid_set(hd.tau));
    adaptive_ = hd.adaptive != 0;
    SG_TRY(enqueue_sort());
    SG_TRY(enqueue_fields());
    SG_CUDA(cudaMemcpyAsync(dd_, &hd.dd, sizeof(DevDiag), cudaMemcpyHostToDevice, stream_));
    SG_CUDA(cudaStreamSynchronize(stream_));
    step_ = hd.step;
    phase_ = kReady;
    invalidate_graphs();
    return check_status();
  }

  int device_particles(sg_particles_out* out) override {
    std::memset(out, 0, sizeof(*out));
    out->n = np_;
    out->on_device = 1;
    for (int m = 0; m < D; ++m) {
      out->u[m] = P_[cur_].u[m];
      out->v[m] = P_[cur_].v[m];
    }
    out->w = P_[cur_].w;
    return SG_OK;
  }

  int set_profiling(int on) override {
    profiling_ = on != 0;
    if (profiling_ && !ev_[0]) {
      for (int i = 0; i < 8; ++i) SG_CUDA(cudaEventCreate(&ev_[i]));
    }
    return SG_OK;
  }

  // Fix the solve variant (0 per-axis passes, 1 one block per grid) or
  // return to autotuning (-1); kept across grid-set changes.
  int set_solve_variant(int variant) override {
    if (variant < -1 || variant > 1) {
      set_error("sg_pic_set_solve_variant: variant must be -1, 0 or 1");
      return SG_ERR_INVALID;
    }
    if (variant == 1 && !small_solve_fits()) {
      set_error("sg_pic_set_solve_variant: a component grid is too large for the one-block solve");
      return SG_ERR_UNSUPPORTED;
    }
    SG_CUDA(cudaStreamSynchronize(stream_));
    invalidate_graphs();
    force_mode_ = variant;
    if (filter_) return SG_OK;  // the filter mode runs no component solves
    return tune_solve();
  }

  int stage_times(double* ms, int cap) override {
    for (int i = 0; i < 6 && i < cap; ++i) ms[i] = stage_ms_[i];
    // autotuner record: chosen solve variant and the timings it compared
    if (cap > 6) ms[6] = solve_mode_;
    if (cap > 7) ms[7] = solve_ms_[0];
    if (cap > 8) ms[8] = solve_ms_[1];
    if (cap > 9) ms[9] = tuned_from_cache_ ? 1.0 : 0.0;
    // particle-pass tuner: push grid in use, one resident wave, the three
    // push timings (half, one, two waves), the window capacity in use, the
    // four deposit timings, and whether they came from the cache
    if (cap > 10) ms[10] = push_blocks_;
    if (cap > 11) ms[11] = push_wave_;
    for (int c = 0; c < kPushCands; ++c)
      if (cap > 12 + c) ms[12 + c] = push_ms_[c];
    if (cap > 15) ms[15] = win_cap_;
    for (int c = 0; c < kDepCands; ++c)
      if (cap > 16 + c) ms[16 + c] = dep_ms_[c];
    if (cap > 20) ms[20] = part_from_cache_ ? 1.0 : 0.0;
    // the deposit timed again before the first sort step (0 until then)
    for (int c = 0; c < kDepCands; ++c)
      if (cap > 21 + c) ms[21 + c] = dep_drift_ms_[c];
    return SG_OK;
  }

  unsigned long long kernel_launches() const override { return launches_; }
  size_t device_bytes() const override { return bytes_; }
  cudaStream_t stream() const override { return stream_; }
  size_t n_particles() const override { return np_; }
  long long steps_done() const override { return step_; }
  bool next_step_sorts() const { return ((step_ + 1) % sort_every_) == 0; }
  int step_plain() override {
    const bool do_sort = next_step_sorts();
    const unsigned long long l0 = launches_so_far();
    per_grid_ = true;
    const int st = enqueue_step(do_sort);
    per_grid_ = false;
    if (st != SG_OK) return st;
    ++step_;
    launches_ += launches_so_far() - l0;
    return SG_OK;
  }

 private:
  // ------------------------------------------------------------ memory
  // Device memory comes from the stream-ordered allocator on the run's
  // stream: freeing does not synchronise the device (a server retiring one
  // run does not stall the others), and the device's pool keeps freed
  // memory for the next run instead of returning it to the driver.
  int alloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(p, bytes, stream_);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
      return SG_ERR_OOM;
    }
    bufs_.push_back({*p, bytes});
    bytes_ += bytes;
    return SG_OK;
  }
  // Once per device in the process: the default pool keeps up to 16 GB of
  // freed memory for reuse (process-local, released at exit).
  static void keep_pool_memory() {
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      unsigned long long keep = 16ull << 30;  // the attribute is a 64-bit unsigned value
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
  }
  void free_one(void* p) {
    if (!p) return;
    for (size_t i = 0; i < bufs_.size(); ++i)
      if (bufs_[i].p == p) {
        cudaFreeAsync(p, stream_);
        bytes_ -= bufs_[i].bytes;
        bufs_.erase(bufs_.begin() + i);
        return;
      }
  }
  void release() {
    invalidate_graphs();
    if (stream_) cudaStreamSynchronize(stream_);
    for (auto& b : bufs_) cudaFreeAsync(b.p, stream_);
    if (stream_) cudaStreamSynchronize(stream_);
    bufs_.clear();
    if (diag_host_) cudaFreeHost(diag_host_);
    diag_host_ = nullptr;
    diag_host_bytes_ = 0;
    if (stats_host_) cudaFreeHost(stats_host_);
    stats_host_ = nullptr;
    stats_host_bytes_ = 0;
    for (auto& r : ring_) {
      if (r.host) cudaFreeHost(r.host);
      if (r.ev) cudaEventDestroy(r.ev);
      r = DiagSlot();
    }
    ring_head_ = ring_count_ = 0;
    for (int i = 0; i < 8; ++i)
      if (ev_[i]) cudaEventDestroy(ev_[i]);
    if (ev_fork_) cudaEventDestroy(ev_fork_);
    if (ev_join_) cudaEventDestroy(ev_join_);
    if (sort_stream_) cudaStreamDestroy(sort_stream_);
    ev_fork_ = ev_join_ = nullptr;
    sort_stream_ = nullptr;
    if (own_stream_ && stream_) cudaStreamDestroy(stream_);
    stream_ = nullptr;
  }
  int size_error(const char* who) {
    set_error(std::string(who) + ": caller buffer too small");
    return SG_ERR_SIZE;
  }
  int copy_to_host_double(const real* src, double* dst, size_t n) {
    double* tmp = nullptr;
    SG_TRY(alloc((void**)&tmp, n * sizeof(double)));
    SG_TRY(launch_to_double<real>(src, tmp, n, stream_));
    SG_CUDA(cudaMemcpyAsync(dst, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, stream_));
    SG_CUDA(cudaStreamSynchronize(stream_));
    free_one(tmp);
    return SG_OK;
  }
  int check_status() {
    unsigned st = 0;
    SG_CUDA(cudaMemcpyAsync(&st, status_, sizeof(unsigned), cudaMemcpyDeviceToHost, stream_));
    SG_CUDA(cudaStreamSynchronize(stream_));
    if (st & ST_NONFINITE) {
      set_error("a kernel produced a non-finite particle state");
      return SG_ERR_NONFINITE;
    }
    return SG_OK;
  }

  int upload_particles(const sg_particles* parts) {
    cudaMemcpyKind kind = parts->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (np_ > 0) {
      for (int m = 0; m < D; ++m) {
        if (!parts->u[m] || !parts->v[m]) {
          set_error("sg_pic_init: NULL particle array");
          return SG_ERR_INVALID;
        }
        SG_CUDA(cudaMemcpyAsync(P_[cur_].u[m], parts->u[m], np_ * sizeof(real), kind, stream_));
        SG_CUDA(cudaMemcpyAsync(P_[cur_].v[m], parts->v[m], np_ * sizeof(real), kind, stream_));
      }
      if (!parts->w) {
        set_error("sg_pic_init: NULL charge array");
        return SG_ERR_INVALID;
      }
      SG_CUDA(cudaMemcpyAsync(P_[cur_].w, parts->w, np_ * sizeof(real), kind, stream_));
      SG_TRY(launch_wrap_check<real, D>(P_[cur_], np_, status_, stream_));
    }
    return SG_OK;  // particle_stats() checks the status and sets the deposit scale
  }

  // Fixed-point scale of the deposit window (FP32 path): with E the least
  // integer such that max_p |q_p| / V <= 2^E (1 - 2^-11), contributions are
  // scaled by 2^(20 - E), so each rounds to at most 2^20 - 2^9 in magnitude
  // and a window of at most 2^11 particles stays below 2^31 - 2^20.
  // Charges do not change during a run; load() recomputes it.
  void set_deposit_scale(double qmax) {
    dep_scale_ = 1.0;
    if (sizeof(real) == 4 && np_ > 0) {
      qmax *= (double)inv_cell_vol();
      int E = 0;
      if (qmax > 0) std::frexp(qmax, &E);  // qmax < 2^E
      if (qmax > std::ldexp(1.0 - 1.0 / 2048.0, E)) ++E;
      const int k = std::max(-126, std::min(127, 20 - E));
      dep_scale_ = std::ldexp(1.0, k);
    }
  }

  // ------------------------------------------------------------ grid set
  int build_grid_set(int tau) {
    invalidate_graphs();
    solve_mode_ = -1;
    tau_ = tau;
    grids_ = combination_grids(D, n_, tau);
    ngrids_ = (int)grids_.size();
    gdesc_.assign(ngrids_, GridDesc{});
    size_t off = 0;
    lmin_ = n_;
    for (int g = 0; g < ngrids_; ++g) {
      GridDesc& d = gdesc_[g];
      std::memset(&d, 0, sizeof(d));
      int sz = 1;
      double vol = 1;
      for (int m = 0; m < 3; ++m) d.l[m] = grids_[g].l[m];
      for (int m = 0; m < D; ++m) {
        sz <<= d.l[m];
        vol *= cfg_.L[m] / (double)(1 << d.l[m]);
        d.kfac[m] = 2.0 * M_PI / cfg_.L[m];
      }
      d.coeff = grids_[g].coeff;
      d.offset = (int)off;
      d.size = sz;
      d.vol = vol;
      off += (size_t)sz;
      lmin_ = std::min(lmin_, d.l[0]);
    }
    S_ = off;
    // (re)allocate arenas
    for (void* p : grid_bufs_) free_one(p);
    grid_bufs_.clear();
    SG_TRY(galloc((void**)&grids_dev_, ngrids_ * sizeof(GridDesc)));
    {  // grids grouped by x level for the combination
      std::vector<int> order;
      std::memset(&levels_, 0, sizeof(levels_));
      for (int l = 0; l <= n_; ++l) {
        levels_.start[l] = (int)order.size();
        for (int g = 0; g < ngrids_; ++g)
          if (gdesc_[g].l[0] == l) order.push_back(g);
      }
      for (int l = n_ + 1; l < 18; ++l) levels_.start[l] = (int)order.size();
      if ((int)order.size() > CB_MAX_GRIDS) {
        set_error("too many component grids for the combination kernel");
        return SG_ERR_UNSUPPORTED;
      }
      int* dev = nullptr;
      SG_TRY(galloc((void**)&dev, order.size() * sizeof(int)));
      SG_CUDA(cudaMemcpyAsync(dev, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, stream_));
      levels_.grid = dev;
    }
    SG_TRY(galloc((void**)&rho_arena_, S_ * sizeof(real)));
    SG_TRY(galloc((void**)&A_, S_ * sizeof(cplx<real>)));
    SG_TRY(galloc((void**)&B_, (size_t)D * S_ * sizeof(cplx<real>)));
    SG_TRY(galloc((void**)&E_arena_, (size_t)D * S_ * sizeof(real)));
    SG_CUDA(cudaMemcpyAsync(grids_dev_, gdesc_.data(), ngrids_ * sizeof(GridDesc), cudaMemcpyHostToDevice, stream_));
    SG_TRY(build_restrict_jobs());
    SG_TRY(build_fft_jobs());
    SG_CUDA(cudaStreamSynchronize(stream_));
    return SG_OK;
  }
  int galloc(void** p, size_t bytes) {
    SG_TRY(alloc(p, bytes));
    grid_bufs_.push_back(*p);
    return SG_OK;
  }

  struct Pass {
    LineJob* dev = nullptr;
    int njobs = 0, nblocks = 0, lpb = 1, vpl = 1, smem = 0;
  };
  struct FPass {
    FftJob* dev = nullptr;
    int kind = 0, njobs = 0, nblocks = 0, smem = 0;
  };

  // Restriction: axis by axis.  Pass a restricts, along axis a, one source
  // array per distinct prefix (l_0 .. l_{a-1}) of the grid set's level
  // vectors, to every level l_a that some grid with that prefix needs.  All
  // arrays keep the natural layout (x fastest): the source of pass a is
  // [outer][N][inner] with inner = the already restricted axes and outer =
  // the axes not reached yet; the last pass writes the component grids.
  int build_restrict_jobs() {
    rpasses_.clear();
    std::map<std::vector<int>, real*> prev;  // arrays of the previous pass
    prev[{}] = rho_reg_;
    int S = N_ + ((N_ >> 5) << 2);  // tile row: 4 padding words per 32, = 4 (mod 32)
    S = (S + 3) & ~3;
    while ((S & 31) != 4) S += 4;
    for (int a = 0; a < D; ++a) {
      std::map<std::vector<int>, std::set<int>> targets;  // prefix -> levels along axis a
      for (auto& g : grids_) {
        std::vector<int> pre(g.l, g.l + a);
        targets[pre].insert(g.l[a]);
      }
      std::vector<LineJob> jobs;
      std::map<std::vector<int>, real*> next;
      long long total_lines = 0;
      for (auto& kv : targets) {
        LineJob J;
        std::memset(&J, 0, sizeof(J));
        J.src = prev.at(kv.first);
        J.sub_mean = J.src == rho_reg_ ? 1 : 0;
        J.top = n_;
        long long inner = 1, outer = 1;
        for (int m = 0; m < a; ++m) inner <<= kv.first[m];
        for (int m = a + 1; m < D; ++m) outer *= N_;
        J.inner = (int)inner;
        J.outer = (int)outer;
        J.tile_stride = S;
        J.tmin = n_;
        for (int tl : kv.second) {
          if (tl < 0 || tl >= RJ_LEVELS) {
            set_error("restriction: level out of range");
            return SG_ERR_UNSUPPORTED;
          }
          std::vector<int> key = kv.first;
          key.push_back(tl);
          if (a < D - 1 && tl == n_) {  // unrestricted along this axis: the source itself, same layout
            next[key] = prev.at(kv.first);
            continue;
          }
          J.tmask |= 1 << tl;
          J.tmin = std::min(J.tmin, tl);
          real* dst;
          if (a == D - 1) {  // final pass writes the component grid
            int gi = find_grid(key);
            dst = rho_arena_ + gdesc_[gi].offset;
          } else {
            SG_TRY(galloc((void**)&dst, ((size_t)outer << tl) * (size_t)inner * sizeof(real)));
            next[key] = dst;
          }
          J.dst[tl] = dst;
        }
        if (J.tmask == 0) continue;  // every target aliases the source
        total_lines += outer * inner;
        jobs.push_back(J);
      }
      if (jobs.empty()) {  // e.g. tau = n: nothing to restrict along this axis
        prev.swap(next);
        continue;
      }
      // lines per block: contiguous lines (pass 0) need no tile, so blocks
      // are sized to cover every SM twice; strided lines take tiles of 8
      // adjacent lines (32-byte row segments) within 160 KB of shared memory
      int lpb = 8;
      if (a == 0) {
        while (lpb > 1 && total_lines / lpb < 2 * 152) lpb >>= 1;
      } else {
        while (lpb > 1 && (size_t)lpb * S * sizeof(real) > 160 * 1024) lpb >>= 1;
      }
      int blocks = 0;
      for (auto& J : jobs) {
        J.block_begin = blocks;
        if (J.inner == 1) {
          blocks += (J.outer + lpb - 1) / lpb;
        } else {
          const int cpb = std::min(lpb, J.inner);
          blocks += J.outer * (J.inner / cpb);
        }
      }
      Pass P;
      P.njobs = (int)jobs.size();
      P.nblocks = blocks;
      P.lpb = lpb;
      P.vpl = std::max(1, N_ / 32);
      P.smem = a == 0 ? 0 : (int)((size_t)lpb * S * sizeof(real));
      SG_TRY(galloc((void**)&P.dev, jobs.size() * sizeof(LineJob)));
      // pageable source: staged when the call returns, no synchronisation needed
      SG_CUDA(cudaMemcpyAsync(P.dev, jobs.data(), jobs.size() * sizeof(LineJob), cudaMemcpyHostToDevice, stream_));
      rpasses_.push_back(P);
      prev.swap(next);
    }
    return SG_OK;
  }
  int find_grid(const std::vector<int>& l) {
    for (int g = 0; g < ngrids_; ++g) {
      bool eq = true;
      for (int m = 0; m < D; ++m) eq &= grids_[g].l[m] == l[m];
      if (eq) return g;
    }
    return -1;
  }

  int build_fft_jobs() {
    fpasses_.clear();
    std::vector<std::pair<int, int>> seq;  // (kind, axis)
    if (D == 2) {
      seq = {{FFT_FWD_FIRST, 0}, {FFT_LAST, 1}, {FFT_INV_LAST, 0}};
    } else {
      seq = {{FFT_FWD_FIRST, 0}, {FFT_FWD_MID, 1}, {FFT_LAST, 2}, {FFT_INV_MID, 1}, {FFT_INV_LAST, 0}};
    }
    const int CAPC = FFT_BLOCK_VALUES;  // complex values per buffer (whole lines, at least one)
    for (auto& ka : seq) {
      const int kind = ka.first, axis = ka.second;
      const bool per_comp = (kind == FFT_INV_MID || kind == FFT_INV_LAST);
      std::vector<FftJob> jobs;
      int blocks = 0, smem = 0;
      for (int g = 0; g < ngrids_; ++g) {
        for (int comp = 0; comp < (per_comp ? (D + 1) / 2 : 1); ++comp) {  // component pairs
          FftJob J;
          std::memset(&J, 0, sizeof(J));
          J.grid = g;
          for (int m = 0; m < 3; ++m) J.dims[m] = m < D ? (1 << gdesc_[g].l[m]) : 1;
          J.axis = axis;
          J.logn = gdesc_[g].l[axis];
          const int len = 1 << J.logn;
          J.lines = gdesc_[g].size / len;
          int C = std::max(1, CAPC / len);
          if (C > J.lines) C = J.lines;
          J.lines_per_block = C;
          J.block_begin = blocks;
          J.comp = comp;
          blocks += (J.lines + C - 1) / C;
          const size_t padded = (size_t)C * len + (((size_t)C * len) >> 5);  // see fpad in the solve
          smem = std::max(smem, (int)(2 * padded * sizeof(cplx<real>)));
          jobs.push_back(J);
        }
      }
      FPass P;
      P.kind = kind;
      P.njobs = (int)jobs.size();
      P.nblocks = blocks;
      P.smem = smem;
      SG_TRY(galloc((void**)&P.dev, jobs.size() * sizeof(FftJob)));
      // pageable source: staged when the call returns, no synchronisation needed
      SG_CUDA(cudaMemcpyAsync(P.dev, jobs.data(), jobs.size() * sizeof(FftJob), cudaMemcpyHostToDevice, stream_));
      fpasses_.push_back(P);
    }
    return SG_OK;
  }

  int ensure_estimator_buffers() {
    if (est_z_) return SG_OK;
    SG_TRY(alloc((void**)&est_rho_, ND_ * sizeof(double)));
    SG_TRY(alloc((void**)&est_z_, ND_ * sizeof(cplx<double>)));
    SG_TRY(alloc((void**)&est_w_, ND_ * sizeof(cplx<double>)));
    SG_TRY(alloc((void**)&est_scalar_, 16 * sizeof(double)));
    const std::vector<cplx<double>> tw = make_twiddles<double>(n_);
    SG_TRY(alloc((void**)&tw64_, tw.size() * sizeof(cplx<double>)));
    SG_CUDA(cudaMemcpyAsync(tw64_, tw.data(), tw.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice, stream_));
    return SG_OK;
  }

  // ------------------------------------------------------------ step stages
  double fe_scale() const {
    double hd = 1;
    for (int m = 0; m < D; ++m) hd *= cfg_.L[m] / (double)N_;
    return 0.5 * hd;
  }
  // Mean charge density Q / |box|: the mean of every component density and
  // of the filtered density (the transfer operators and the deposit conserve
  // the total charge).  The restriction subtracts it as it reads the regular
  // grid, so the component densities and the filtered density are stored as
  // deviations from it; the getters and the charge diagnostics add the
  // same value back in FP64.
  real rho_mean() const { return (real)(charge_total_ / box_volume()); }
  double box_volume() const {
    double vol = 1;
    for (int m = 0; m < D; ++m) vol *= cfg_.L[m];
    return vol;
  }
  int add_mean(double* rho, size_t n) const {
    const double mean = (double)rho_mean();
    for (size_t i = 0; i < n; ++i) rho[i] += mean;
    return SG_OK;
  }
  real inv_cell_vol() const {
    double hd = 1;
    for (int m = 0; m < D; ++m) hd *= cfg_.L[m] / (double)N_;
    return (real)(1.0 / hd);
  }

  int enqueue_push(double dt, bool drift, double* ke, bool fuse_sort = false) {
    PushParams<real> pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.qm = (real)cfg_.qm;
    pp.dt = (real)dt;
    pp.ke_fac = (real)(0.5 / cfg_.qm);
    bool boris = false, eext = false;
    for (int m = 0; m < 3; ++m) {
      pp.dt_over_L[m] = m < D ? (real)(dt / cfg_.L[m]) : (real)0;
      pp.eext[m] = m < D ? (real)(cfg_.eext_lin[m] * cfg_.L[m]) : (real)0;
      pp.tB[m] = (real)(cfg_.qm * cfg_.B[m] * 0.5 * dt);
      boris |= cfg_.B[m] != 0.0;
      eext |= (m < D && cfg_.eext_lin[m] != 0.0);
    }
    pp.boris = boris ? 1 : 0;
    pp.has_eext = eext ? 1 : 0;
    pp.drift = drift ? 1 : 0;
    pp.shift = cfg_.cell ? (real)0.5 : (real)0;
    SortFuse sf;
    if (fuse_sort) {
      SG_TRY(sort_reset());
      sf = sort_fuse();
    }
    return launch_push<real, D>(P_[cur_], np_, n_, Ehi_, pp, ke, status_, sf, stream_, push_blocks_);
  }

  // Step sort: counting sort of the particles by tile key (the Morton key of
  // the level-(n - tile_shift) cell), in two halves: keys + tile counts
  // (emitted by the push on sort steps, or by k_tile_keys), then the scan of
  // the counts and one scatter pass of the particle payload.
  SortFuse sort_fuse() const {
    SortFuse sf;
    sf.keys = keys_;
    sf.checksum = checksum_;
    sf.tile_shift = tile_shift_;
    return sf;
  }
  int sort_reset() {
    SG_CUDA(cudaMemsetAsync(checksum_, 0, sizeof(unsigned long long), stream_));
    SG_CUDA(cudaMemsetAsync(tile_count_, 0, ntiles_ * sizeof(uint32_t), stream_));
    return SG_OK;
  }
  int sort_finish(cudaStream_t s = nullptr) {
    if (!s) s = stream_;
    SG_TRY(launch_tile_hist(keys_, np_, tile_count_, s));
    SG_TRY(exclusive_scan_u32(tile_count_, cursor_, ntiles_, scan_sums_, s));
    SG_TRY(launch_tile_scatter<real, D>(P_[cur_], P_[cur_ ^ 1], keys_, cursor_, np_, s));
    cur_ ^= 1;
    return SG_OK;
  }
  int enqueue_sort() {  // from the current positions (init, load)
    SG_TRY(sort_reset());
    SG_TRY(launch_tile_keys<real, D>(P_[cur_], np_, n_, sort_fuse(), status_, stream_));
    return sort_finish();
  }

  int enqueue_deposit() {
    SG_CUDA(cudaMemsetAsync(rho_reg_, 0, ND_ * sizeof(real), stream_));
    return launch_deposit<real, D>(P_[cur_], np_, n_, inv_cell_vol(), rho_reg_, win_cap_, (real)dep_scale_,
                                   (real)(1.0 / dep_scale_), cfg_.cell ? (real)0.5 : (real)0, stream_);
  }

  int enqueue_restrict() {
    for (auto& P : rpasses_)
      SG_TRY(launch_restrict_pass<real>(P.dev, P.njobs, P.nblocks, P.lpb, P.vpl, P.smem, cfg_.cell, rho_mean(),
                                        stream_));
    return SG_OK;
  }

  SolveArena<real> solve_arena() const {
    SolveArena<real> a;
    a.grids = grids_dev_;
    a.rho = rho_arena_;
    a.A = A_;
    a.B = B_;
    a.E = E_arena_;
    a.S = S_;
    a.tw = tw_;
    a.log_nmax = n_;
    a.dim = D;
    return a;
  }
  int enqueue_solve() {
    const SolveArena<real> a = solve_arena();
    int maxsize = 0;
    for (auto& g : gdesc_) maxsize = std::max(maxsize, g.size);
    const bool small_ok = maxsize <= small_solve_max<real>();
    if (small_ok && per_grid_) {  // plain path: one launch per component grid
      for (int g = 0; g < ngrids_; ++g) SG_TRY(launch_solve_small<real>(a, 1, gdesc_[g].size, stream_, g));
      return SG_OK;
    }
    if (small_ok && solve_mode_ == 1) return launch_solve_small<real>(a, ngrids_, maxsize, stream_);
    for (auto& P : fpasses_) SG_TRY(launch_fft_pass<real>(P.kind, a, P.dev, P.njobs, P.nblocks, P.smem, stream_));
    return SG_OK;
  }

  // Autotuning of the solve: time the one-block-per-grid kernel against the
  // per-axis passes on this grid set (both read the component densities and
  // write the component fields, so repeating them is harmless) and keep the
  // faster.  Runs at init and whenever the grid set changes.
  bool small_solve_fits() const {
    int maxsize = 0;
    for (auto& g : gdesc_) maxsize = std::max(maxsize, g.size);
    return maxsize <= small_solve_max<real>();
  }

  int tune_solve() {
    if (!small_solve_fits()) {
      solve_mode_ = 0;
      return SG_OK;
    }
    if (force_mode_ >= 0) {  // fixed by the caller: no timing
      solve_mode_ = force_mode_;
      return SG_OK;
    }
    // The choice depends only on the grid set and the precision: a run with
    // the same (precision, d, n, tau) as an earlier one in this process
    // takes the earlier timing instead of repeating it.
    const TuneKey key{(int)sizeof(real), D, n_, tau_};
    {
      std::lock_guard<std::mutex> lk(tune_mu());
      auto it = tune_cache().find(key);
      if (it != tune_cache().end()) {
        solve_mode_ = it->second.mode;
        solve_ms_[0] = it->second.ms[0];
        solve_ms_[1] = it->second.ms[1];
        tuned_from_cache_ = true;
        return SG_OK;
      }
    }
    tuned_from_cache_ = false;
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0));
    SG_CUDA(cudaEventCreate(&e1));
    float best[2] = {1e30f, 1e30f};
    for (int rep = 0; rep < 3; ++rep) {
      for (int mode = 0; mode < 2; ++mode) {
        solve_mode_ = mode;
        SG_CUDA(cudaEventRecord(e0, stream_));
        SG_TRY(enqueue_solve());
        SG_CUDA(cudaEventRecord(e1, stream_));
        SG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        SG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best[mode] = std::min(best[mode], ms);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    solve_mode_ = best[1] < best[0] ? 1 : 0;
    solve_ms_[0] = best[0];
    solve_ms_[1] = best[1];
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_cache()[key] = TuneEntry{solve_mode_, {best[0], best[1]}};
    return SG_OK;
  }

  // Particle-pass autotuner, run once per run shape in the process (the
  // choice is cached like the solve variant's): the push's grid -- half,
  // one or two resident waves of blocks, i.e. the particles per block -- and
  // the deposit's window capacity, which sets the window's side (its tile
  // of the regular grid) and how many windows fit on an SM.  Both are timed
  // on the run's own particles and leave the state as it was: the push runs
  // with dt = 0 (every increment is an exact zero, so the particles stay
  // bit for bit), the deposit recomputes the regular-grid density of the
  // same particles.  The deposit is timed on freshly sorted particles (its
  // best case).  A candidate replaces the default only when it is at least
  // 3% faster, so that timing noise does not move the choice.
  int tune_particles() {
    if (np_ == 0) return SG_OK;
    bool boris = false;
    for (int m = 0; m < 3; ++m) boris |= cfg_.B[m] != 0.0;
    int lg = 0;
    while (((size_t)1 << (lg + 1)) <= np_) ++lg;
    const PartKey key{(int)sizeof(real), D, n_, lg, cfg_.cell ? 1 : 0, boris ? 1 : 0};
    const int pcand[kPushCands] = {std::max(1, push_wave_ / 2), push_wave_, 2 * push_wave_};
    auto apply = [&](int pp, int dp) {
      push_pick_ = pp;
      dep_pick_ = dp;
      push_blocks_ = pcand[pp];
      nke_ = push_blocks_;
      win_cap_ = kDepCap[dp];
    };
    {
      std::lock_guard<std::mutex> lk(tune_mu());
      auto it = part_cache().find(key);
      if (it != part_cache().end()) {
        for (int c = 0; c < kPushCands; ++c) push_ms_[c] = it->second.push_ms[c];
        for (int c = 0; c < kDepCands; ++c) dep_ms_[c] = it->second.dep_ms[c];
        for (int c = 0; c < kDepCands; ++c) dep_drift_ms_[c] = it->second.dep_drift_ms[c];
        apply(it->second.push_pick, it->second.dep_pick);
        part_from_cache_ = true;
        refine_pending_ = !it->second.refined;
        return SG_OK;
      }
    }
    part_from_cache_ = false;
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0));
    SG_CUDA(cudaEventCreate(&e1));
    auto timed = [&](auto&& enqueue, float* best) -> int {
      SG_CUDA(cudaEventRecord(e0, stream_));
      SG_TRY(enqueue());
      SG_CUDA(cudaEventRecord(e1, stream_));
      SG_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      SG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      *best = std::min(*best, ms);
      return SG_OK;
    };
    float pms[kPushCands], dms[kDepCands];
    for (int rep = 0; rep < 4; ++rep) {  // the first round warms up
      for (int c = 0; c < kPushCands; ++c) {
        if (rep == 0) pms[c] = 1e30f;
        push_blocks_ = pcand[c];
        float warm = 1e30f;
        SG_TRY(timed([&] { return enqueue_push(0.0, true, ke_partials_); }, rep ? &pms[c] : &warm));
      }
      for (int c = 0; c < kDepCands; ++c) {
        if (rep == 0) dms[c] = 1e30f;
        win_cap_ = kDepCap[c];
        float warm = 1e30f;
        SG_TRY(timed([&] { return enqueue_deposit(); }, rep ? &dms[c] : &warm));
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int pp = 1, dp = 2;  // the defaults: one wave, 8192 nodes
    for (int c = 0; c < kPushCands; ++c)
      if (pms[c] < 0.97f * pms[pp]) pp = c;
    for (int c = 0; c < kDepCands; ++c)
      if (dms[c] < 0.97f * dms[dp]) dp = c;
    for (int c = 0; c < kPushCands; ++c) push_ms_[c] = pms[c];
    for (int c = 0; c < kDepCands; ++c) dep_ms_[c] = dms[c];
    apply(pp, dp);
    SG_TRY(enqueue_deposit());  // the regular-grid density from the chosen window
    PartEntry ent;
    std::memset(&ent, 0, sizeof(ent));
    ent.push_pick = pp;
    ent.dep_pick = dp;
    for (int c = 0; c < kPushCands; ++c) ent.push_ms[c] = pms[c];
    for (int c = 0; c < kDepCands; ++c) ent.dep_ms[c] = dms[c];
    ent.refined = false;
    std::lock_guard<std::mutex> lk(tune_mu());
    part_cache()[key] = ent;
    refine_pending_ = true;
    return SG_OK;
  }

  // The second look at the deposit window, just before the run's first sort
  // step: the particles have drifted for a whole sort period since the
  // init sort, the deposit's worst case, where the first timing saw its best.
  // Every candidate is timed again on the current particles (the regular-grid
  // density of unchanged positions is recomputed; the next step recomputes
  // it anyway), and the window minimising the sum of the two timings is
  // kept (3% rule as before).  A change re-captures the step graphs.  The
  // refined choice goes to the cache, so runs of the same shape skip this.
  int refine_deposit() {
    refine_pending_ = false;
    if (np_ == 0 || adaptive_ || profiling_) return SG_OK;
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0));
    SG_CUDA(cudaEventCreate(&e1));
    float dms[kDepCands];
    const int keep = win_cap_;
    int st = SG_OK;
    for (int rep = 0; rep < 3 && st == SG_OK; ++rep) {  // the first round warms up
      for (int c = 0; c < kDepCands && st == SG_OK; ++c) {
        if (rep == 0) dms[c] = 1e30f;
        win_cap_ = kDepCap[c];
        if (cudaEventRecord(e0, stream_) != cudaSuccess) st = SG_ERR_CUDA;
        if (st == SG_OK) st = enqueue_deposit();
        if (st == SG_OK && cudaEventRecord(e1, stream_) != cudaSuccess) st = SG_ERR_CUDA;
        if (st == SG_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SG_ERR_CUDA;
        float ms = 0;
        if (st == SG_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = SG_ERR_CUDA;
        if (st == SG_OK && rep > 0) dms[c] = std::min(dms[c], ms);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    win_cap_ = keep;
    if (st != SG_OK) {
      set_error("deposit window refinement: CUDA error");
      return st;
    }
    int dp = dep_pick_;
    for (int c = 0; c < kDepCands; ++c)
      if (dep_ms_[c] + dms[c] < 0.97f * (dep_ms_[dp] + dms[dp])) dp = c;
    for (int c = 0; c < kDepCands; ++c) dep_drift_ms_[c] = dms[c];
    if (dp != dep_pick_) {
      dep_pick_ = dp;
      win_cap_ = kDepCap[dp];
      invalidate_graphs();
    }
    SG_TRY(enqueue_deposit());  // the regular-grid density from the chosen window
    bool boris = false;
    for (int m = 0; m < 3; ++m) boris |= cfg_.B[m] != 0.0;
    int lg = 0;
    while (((size_t)1 << (lg + 1)) <= np_) ++lg;
    const PartKey key{(int)sizeof(real), D, n_, lg, cfg_.cell ? 1 : 0, boris ? 1 : 0};
    std::lock_guard<std::mutex> lk(tune_mu());
    auto it = part_cache().find(key);
    if (it != part_cache().end()) {
      it->second.dep_pick = dp;
      it->second.refined = true;
      for (int c = 0; c < kDepCands; ++c) it->second.dep_drift_ms[c] = dms[c];
    }
    return SG_OK;
  }

  // The combination's last block also closes the step's FP64 bookkeeping
  // (field energy, previous field energy, kinetic energy of the push when
  // ke is given) unless finalize is false.
  int enqueue_combine(bool finalize = true, const double* ke = nullptr) {
    CombineFinal fin;
    fin.active = finalize ? 1 : 0;
    fin.ke_partials = ke;
    fin.n_ke = nke_;
    fin.fe_scale = fe_scale();
    fin.dd = dd_;
    fin.counter = comb_counter_;
    return launch_combine<real, D>(grids_dev_, levels_, lmin_, E_arena_, S_, n_, Ehi_, Elo_, fe_partials_, fin,
                                   stream_, D, cfg_.cell, cfg_.combine_fp64);
  }

  // Filter mode (Algorithm 2): rho_f = sum_i c_i P_i R_i rho~ on the regular
  // nodes (the combination kernel on the component densities), then one
  // spectral solve there; closes the step's FP64 bookkeeping.
  int enqueue_filter_density() {
    CombineFinal off;
    std::memset(&off, 0, sizeof(off));
    return launch_combine<real, D>(grids_dev_, levels_, lmin_, rho_arena_, S_, n_, rho_f_, nullptr, fe_partials_, off,
                                   stream_, 1, cfg_.cell, cfg_.combine_fp64);
  }
  int enqueue_regular_solve(const double* ke) {
    SG_TRY(launch_regular_solve<real>(rho_f_, regA_, regB_, ktab_, tw_, D, n_, Ehi_, Elo_,
                                      ec_stride<D>(), reg_partials_, reg_blocks_, stream_));
    return launch_finalize_step(reg_partials_, reg_blocks_ * ((D + 1) / 2), ke, ke ? nke_ : 0, fe_scale(), dd_,
                                stream_);
  }
  int enqueue_filter_field(const double* ke) {
    SG_TRY(enqueue_filter_density());
    return enqueue_regular_solve(ke);
  }

  int enqueue_restrict_solve_combine(const double* ke = nullptr) {
    if (filter_) {
      SG_TRY(enqueue_restrict());
      return enqueue_filter_field(ke);
    }
    SG_TRY(enqueue_restrict());
    SG_TRY(enqueue_solve());
    return enqueue_combine(true, ke);
  }

  int enqueue_fields(const double* ke = nullptr) {
    SG_TRY(enqueue_deposit());
    return enqueue_restrict_solve_combine(ke);
  }

  // A sort step deposits the particles in their current order; then a
  // second stream sorts them into the other buffer (tile counts, scan,
  // scatter: memory-bound) while the latency-bound grid stages, which leave
  // most SMs idle, run on the run's stream; the next step starts from the
  // sorted buffer.  The deposit needs no sorted input: the sort only makes
  // later deposits and gathers faster.
  int enqueue_step(bool do_sort) {
    SG_TRY(enqueue_push(cfg_.dt, true, ke_partials_, do_sort));
    if (!do_sort) return enqueue_fields(ke_partials_);
    SG_TRY(enqueue_deposit());  // P_[cur_]: before sort_finish switches cur_
    SG_CUDA(cudaEventRecord(ev_fork_, stream_));
    SG_CUDA(cudaStreamWaitEvent(sort_stream_, ev_fork_, 0));
    SG_TRY(sort_finish(sort_stream_));  // P_[cur_] -> P_[cur_ ^ 1]
    SG_CUDA(cudaEventRecord(ev_join_, sort_stream_));
    SG_TRY(enqueue_restrict_solve_combine(ke_partials_));
    SG_CUDA(cudaStreamWaitEvent(stream_, ev_join_, 0));
    return SG_OK;
  }

  // Graph variants: (current particle set, sort or not).
  int step_graph(bool do_sort) {
    int vi = cur_ * 2 + (do_sort ? 1 : 0);
    if (!gexec_[vi]) {
      int cur_before = cur_;
      unsigned long long l0 = launches_so_far();
      cudaGraph_t g;
      SG_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
      int st = enqueue_step(do_sort);
      cudaError_t e = cudaStreamEndCapture(stream_, &g);
      cur_ = cur_before;  // the capture did not run anything
      if (st != SG_OK) return st;
      if (e != cudaSuccess) {
        set_error(std::string("graph capture: ") + cudaGetErrorString(e));
        return SG_ERR_CUDA;
      }
      SG_CUDA(cudaGraphInstantiate(&gexec_[vi], g, 0));
      cudaGraphDestroy(g);
      glaunches_[vi] = launches_so_far() - l0;
    }
    SG_CUDA(cudaGraphLaunch(gexec_[vi], stream_));
    launches_ += glaunches_[vi];
    if (do_sort) cur_ ^= 1;
    return SG_OK;
  }

  void invalidate_graphs() {
    for (int i = 0; i < 4; ++i) {
      if (gexec_[i]) {
        cudaGraphExecDestroy(gexec_[i]);
        gexec_[i] = nullptr;
      }
      if (gpre_[i]) {
        cudaGraphExecDestroy(gpre_[i]);
        gpre_[i] = nullptr;
      }
    }
    if (gpost_) {
      cudaGraphExecDestroy(gpost_);
      gpost_ = nullptr;
    }
  }

  // Captures what `enqueue` launches on the run's stream into an executable
  // graph; *launches receives the kernel count.
  template <typename F>
  int capture(F&& enqueue, cudaGraphExec_t* exec, unsigned long long* launches) {
    const int cur_before = cur_;
    const unsigned long long l0 = launches_so_far();
    cudaGraph_t g;
    SG_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
    const int st = enqueue();
    const cudaError_t e = cudaStreamEndCapture(stream_, &g);
    cur_ = cur_before;  // the capture did not run anything
    if (st != SG_OK) return st;
    if (e != cudaSuccess) {
      set_error(std::string("graph capture: ") + cudaGetErrorString(e));
      return SG_ERR_CUDA;
    }
    SG_CUDA(cudaGraphInstantiate(exec, g, 0));
    cudaGraphDestroy(g);
    *launches = launches_so_far() - l0;
    return SG_OK;
  }

  // ------------------------------------------------------------ cross-run solve
  // The step split around the component solves, so that a server can solve
  // the grids of all its resident runs in one launch (launch_solve_batch):
  // step_pre (push, sort when due, deposit, restriction), the caller's
  // solve over solve_jobs, then step_post (combination and the step's FP64
  // bookkeeping).  Runs of the combination mode with a fixed tau whose grids
  // all fit one block take part.
  bool solve_batchable() const override {
    return !adaptive_ && !filter_ && !profiling_ && phase_ == kReady && small_solve_fits();
  }
  int real_bytes() const override { return (int)sizeof(real); }
  int enqueue_step_pre(bool do_sort) {
    SG_TRY(enqueue_push(cfg_.dt, true, ke_partials_, do_sort));
    if (do_sort) SG_TRY(sort_finish());
    SG_TRY(enqueue_deposit());
    return enqueue_restrict();
  }
  int step_pre() override {
    if (!solve_batchable()) {
      set_error("step_pre: the run cannot take part in a cross-run solve");
      return SG_ERR_STATE;
    }
    const bool do_sort = next_step_sorts();
    const int vi = cur_ * 2 + (do_sort ? 1 : 0);
    if (!gpre_[vi]) SG_TRY(capture([&] { return enqueue_step_pre(do_sort); }, &gpre_[vi], &gpre_launches_[vi]));
    SG_CUDA(cudaGraphLaunch(gpre_[vi], stream_));
    launches_ += gpre_launches_[vi];
    if (do_sort) cur_ ^= 1;
    phase_ = kPreSolve;
    return SG_OK;
  }
  int solve_jobs(std::vector<unsigned char>& out, int* max_size, int* max_log) override {
    if (phase_ != kPreSolve) {
      set_error("solve_jobs: step_pre must come first");
      return SG_ERR_STATE;
    }
    const SolveArena<real> a = solve_arena();
    for (int g = 0; g < ngrids_; ++g) {
      SolveJob<real> j;
      std::memset(&j, 0, sizeof(j));
      j.a = a;
      j.grid = g;
      const unsigned char* b = reinterpret_cast<const unsigned char*>(&j);
      out.insert(out.end(), b, b + sizeof(j));
      *max_size = std::max(*max_size, gdesc_[g].size);
    }
    *max_log = std::max(*max_log, n_);
    return SG_OK;
  }
  int step_post() override {
    if (phase_ != kPreSolve) {
      set_error("step_post: step_pre must come first");
      return SG_ERR_STATE;
    }
    if (!gpost_) SG_TRY(capture([&] { return enqueue_combine(true, ke_partials_); }, &gpost_, &gpost_launches_));
    SG_CUDA(cudaGraphLaunch(gpost_, stream_));
    launches_ += gpost_launches_ + 1;  // and this run's share of the cross-run solve
    ++step_;
    phase_ = kReady;
    return SG_OK;
  }

  // Same sequence as enqueue_step with events between the stages:
  // 0 push, 1 sort, 2 deposit, 3 restrict, 4 solve, 5 combine (+ finalize).
  int step_profiled(bool do_sort) {
    unsigned long long l0 = launches_so_far();
    SG_CUDA(cudaEventRecord(ev_[0], stream_));
    SG_TRY(enqueue_push(cfg_.dt, true, ke_partials_, do_sort));
    SG_CUDA(cudaEventRecord(ev_[1], stream_));
    if (do_sort) SG_TRY(sort_finish());
    SG_CUDA(cudaEventRecord(ev_[2], stream_));
    SG_TRY(enqueue_deposit());
    SG_CUDA(cudaEventRecord(ev_[3], stream_));
    SG_TRY(enqueue_restrict());
    SG_CUDA(cudaEventRecord(ev_[4], stream_));
    if (filter_) {  // 4: the density filter, 5: the regular-grid solve
      SG_TRY(enqueue_filter_density());
      SG_CUDA(cudaEventRecord(ev_[5], stream_));
      SG_TRY(enqueue_regular_solve(ke_partials_));
    } else {
      SG_TRY(enqueue_solve());
      SG_CUDA(cudaEventRecord(ev_[5], stream_));
      SG_TRY(enqueue_combine(true, ke_partials_));
    }
    SG_CUDA(cudaEventRecord(ev_[6], stream_));
    SG_CUDA(cudaEventSynchronize(ev_[6]));
    for (int i = 0; i < 6; ++i) {
      float ms = 0;
      SG_CUDA(cudaEventElapsedTime(&ms, ev_[i], ev_[i + 1]));
      stage_ms_[i] += ms;
    }
    launches_ += launches_so_far() - l0;
    return SG_OK;
  }

  int step_adaptive(bool do_sort) {
    unsigned long long l0 = launches_so_far();
    SG_TRY(enqueue_push(cfg_.dt, true, ke_partials_, do_sort));
    if (do_sort) SG_TRY(sort_finish());
    SG_TRY(enqueue_deposit());
    int t = tau_;
    int st = select_tau(&t, nullptr, nullptr, 0);
    if (st == SG_OK && t != tau_) {
      SG_CUDA(cudaStreamSynchronize(stream_));
      SG_TRY(build_grid_set(t));
    } else if (st != SG_OK && st != SG_ERR_RANGE) {
      return st;
    }
    SG_TRY(enqueue_restrict_solve_combine(ke_partials_));
    launches_ += launches_so_far() - l0;
    return SG_OK;
  }

  // ------------------------------------------------------------ state
  enum Phase { kReady = 0, kAwaitStart = 1, kHalfStep = 2, kPreSolve = 3 };
  Phase phase_ = kReady;
  EngineConfig cfg_;
  int n_ = 0, N_ = 0;
  size_t ND_ = 0, np_ = 0, S_ = 0;
  cudaStream_t stream_ = nullptr;
  bool own_stream_ = false;
  int sort_every_ = 1;
  int tau_ = 1;
  bool adaptive_ = false;
  long long step_ = 0;
  double charge_total_ = 0;

  std::vector<DevBuf> bufs_;
  std::vector<void*> grid_bufs_;
  size_t bytes_ = 0;

  PArrays<real, D> P_[2];
  int cur_ = 0;
  uint32_t *keys_ = nullptr, *keys_alt_ = nullptr;
  uint32_t *tile_count_ = nullptr, *cursor_ = nullptr, *scan_sums_ = nullptr;
  int tile_shift_ = 0;
  size_t ntiles_ = 1;
  DevDiag* dd_ = nullptr;
  unsigned* status_ = nullptr;
  unsigned long long* checksum_ = nullptr;
  double* ke_partials_ = nullptr;
  double* fe_partials_ = nullptr;
  unsigned* comb_counter_ = nullptr;
  double dep_scale_ = 1.0;  // FP32 deposit window: fixed-point scale (power of two)
  // filter mode (Algorithm 2): filtered density, regular-grid transform buffers
  bool filter_ = false;
  real* rho_f_ = nullptr;
  cplx<real>* regA_ = nullptr;
  cplx<real>* regB_ = nullptr;
  real* ktab_ = nullptr;
  double* reg_partials_ = nullptr;
  int reg_blocks_ = 0;
  int nke_ = 0, nrows_ = 0;
  // particle-pass tuner: the push grid (one resident wave, and the count in
  // use), the deposit window capacity in use, the compared timings (ms)
  int push_wave_ = 1, push_blocks_ = 1, win_cap_ = 8192;
  int push_pick_ = 1, dep_pick_ = 2;
  float push_ms_[kPushCands] = {}, dep_ms_[kDepCands] = {};
  bool part_from_cache_ = false;
  bool refine_pending_ = false;  // the deposit window is re-timed before the first sort step
  // the sort of a sort step runs on its own stream, forked from and joined
  // to the run's stream (captured into the step graph with it)
  cudaStream_t sort_stream_ = nullptr;
  cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
  float dep_drift_ms_[kDepCands] = {};

  real* rho_reg_ = nullptr;
  real* Ehi_ = nullptr;
  float* Elo_ = nullptr;
  cplx<real>* tw_ = nullptr;

  std::vector<GridSpec> grids_;
  std::vector<GridDesc> gdesc_;
  int ngrids_ = 0, lmin_ = 0;
  LevelLists levels_{};
  bool per_grid_ = false;
  int solve_mode_ = -1;  // -1 untuned, 0 per-axis passes, 1 one block per grid
  int force_mode_ = -1;  // solve variant fixed by the caller, -1 autotuned
  float solve_ms_[2] = {0, 0};
  bool tuned_from_cache_ = false;
  GridDesc* grids_dev_ = nullptr;
  void* diag_host_ = nullptr;  // pinned staging of the diagnostics read-back
  size_t diag_host_bytes_ = 0;
  void* stats_host_ = nullptr;  // mapped pinned: the upload's statistics (particle_stats)
  size_t stats_host_bytes_ = 0;
  static constexpr int kDiagRing = SG_DIAG_RING;
  struct DiagSlot {
    void* host = nullptr;  // pinned record (diag_bytes() at the post)
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;  // recorded after the record's copies
    DiagMeta meta;
  };
  DiagSlot ring_[kDiagRing];
  int ring_head_ = 0, ring_count_ = 0;
  real* rho_arena_ = nullptr;
  cplx<real>* A_ = nullptr;
  cplx<real>* B_ = nullptr;
  real* E_arena_ = nullptr;
  std::vector<Pass> rpasses_;
  std::vector<FPass> fpasses_;

  double* est_rho_ = nullptr;
  cplx<double>* est_z_ = nullptr;
  cplx<double>* est_w_ = nullptr;
  double* est_scalar_ = nullptr;
  cplx<double>* tw64_ = nullptr;

  cudaGraphExec_t gexec_[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned long long glaunches_[4] = {0, 0, 0, 0};
  // the step split around the cross-run solve: (particle set, sort) before
  // the solve, the combination after it
  cudaGraphExec_t gpre_[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned long long gpre_launches_[4] = {0, 0, 0, 0};
  cudaGraphExec_t gpost_ = nullptr;
  unsigned long long gpost_launches_ = 0;
  unsigned long long launches_ = 0;
  bool profiling_ = false;
  cudaEvent_t ev_[8] = {};
  double stage_ms_[6] = {0, 0, 0, 0, 0, 0};
};

}  // namespace

EngineBase* make_engine(int precision, int dim) {
  if (precision == SG_FP32 && dim == 2) return new Engine<float, 2>();
  if (precision == SG_FP32 && dim == 3) return new Engine<float, 3>();
  if (precision == SG_FP64 && dim == 2) return new Engine<double, 2>();
  if (precision == SG_FP64 && dim == 3) return new Engine<double, 3>();
  return nullptr;
}

size_t estimate_footprint(int precision, int dim, int n, int tau, size_t np) {
  size_t rs = precision == SG_FP64 ? 8 : 4;
  size_t ND = (size_t)1 << (dim * n);
  auto grids = combination_grids(dim, n, tau);
  size_t S = 0;
  for (auto& g : grids) {
    size_t s = 1;
    for (int m = 0; m < dim; ++m) s <<= g.l[m];
    S += s;
  }
  size_t part = 2 * np * ((2 * dim + 1) * rs + 4) + 4 * np * 4 + (np / RS_TILE + 1) * 256 * 4 * 2;
  size_t grid = ND * rs * (1 + dim) + (rs == 4 ? dim * ND * 4 : 0) + 2 * ND * rs;  // rho, Ecomb, restrict scratch
  size_t arena = S * (rs + 2 * rs + dim * 2 * rs + dim * rs);
  return part + grid + arena + (1 << 20);
}

}  // namespace sg
