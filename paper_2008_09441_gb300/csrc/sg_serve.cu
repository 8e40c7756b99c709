// Serving: many independent runs resident on one GPU, admitted in arrival
// order by device-memory footprint, advanced together tick by tick.
//
// Batched mode (default): a tick forks from the server's stream into every
// resident run's stream, where the run launches its cached step graph (the
// runs' kernels overlap on the device), and joins back.  Plain mode: each
// run steps in turn with direct kernel launches and one solve launch per
// component grid, each run's step waiting for the previous run's (the
// per-grid, per-run launch path).
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sg_engine.cuh"

using namespace sg;

namespace {

struct Request {
  unsigned long long ticket = 0;
  sg_request req;
  std::vector<char> u[3], v[3], w;  // host copies until admission
  size_t footprint = 0;
  int state = SG_REQ_QUEUED;
  EngineBase* eng = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // timing
  int steps_left = 0;
  sg_diag last{};
  std::vector<char> result_u[3], result_v[3], result_w;
};

}  // namespace

struct sg_server {
  size_t budget = 0;
  int max_slots = 0;
  int mode = SG_SERVE_BATCHED;
  size_t in_use = 0;
  unsigned long long next_ticket = 1;
  std::deque<Request*> queue;
  std::vector<Request*> resident;
  std::map<unsigned long long, Request*> all;
  std::vector<double> step_ms;
  double device_ms = 0;
  double particle_steps = 0;
  unsigned long long steps_served = 0;
  cudaStream_t ds = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // timing
  cudaEvent_t fork = nullptr;                        // start of a tick for the runs' streams (not timed)
  cudaEvent_t solved = nullptr;                      // the cross-run solve of a tick is done (not timed)
  // cross-run solve: job tables per precision (0 FP32, 1 FP64), staged in
  // pinned memory and copied to the device on the server's stream
  void* jobs_dev[2] = {nullptr, nullptr};
  void* jobs_host[2] = {nullptr, nullptr};
  size_t jobs_cap[2] = {0, 0};
  unsigned long long solve_launches = 0, solve_grids = 0;
  std::mutex mu;
};

static int serr(const char* m, int code = SG_ERR_INVALID) {
  set_error(m);
  return code;
}

static void finish(sg_server* s, Request* r, int state) {
  if (r->eng) {
    size_t rs = r->req.params.precision == SG_FP64 ? 8 : 4;
    size_t np = r->req.particles.n;
    int d = r->req.dim;
    for (int m = 0; m < d; ++m) {
      r->result_u[m].resize(np * rs);
      r->result_v[m].resize(np * rs);
    }
    r->result_w.resize(np * rs);
    sg_particles_out o;
    std::memset(&o, 0, sizeof(o));
    o.n = np;
    o.on_device = 0;
    for (int m = 0; m < d; ++m) {
      o.u[m] = r->result_u[m].data();
      o.v[m] = r->result_v[m].data();
    }
    o.w = r->result_w.data();
    if (state == SG_REQ_DONE && r->eng->get_particles(&o) != SG_OK) state = SG_REQ_FAILED;
    r->eng->diagnostics(&r->last);
    delete r->eng;
    r->eng = nullptr;
  }
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
  if (r->stream) cudaStreamDestroy(r->stream);
  r->ev0 = r->ev1 = nullptr;
  r->stream = nullptr;
  for (int m = 0; m < 3; ++m) {
    std::vector<char>().swap(r->u[m]);
    std::vector<char>().swap(r->v[m]);
  }
  std::vector<char>().swap(r->w);
  s->in_use -= r->footprint;
  r->state = state;
}

static int admit(sg_server* s, bool* changed, int* failed) {
  while (!s->queue.empty() && (int)s->resident.size() < s->max_slots &&
         s->in_use + s->queue.front()->footprint <= s->budget) {
    Request* r = s->queue.front();
    s->queue.pop_front();
    s->in_use += r->footprint;
    *changed = true;
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&r->ev0) != cudaSuccess || cudaEventCreate(&r->ev1) != cudaSuccess) {
      finish(s, r, SG_REQ_FAILED);
      continue;
    }
    EngineConfig cfg;
    const sg_request& q = r->req;
    cfg.dim = q.dim;
    cfg.n = q.level_n;
    cfg.tau = q.params.tau;
    cfg.precision = q.params.precision;
    for (int m = 0; m < 3; ++m) {
      cfg.L[m] = m < q.dim ? q.domain.L[m] : 1.0;
      cfg.B[m] = q.params.B[m];
      cfg.eext_lin[m] = q.params.Eext_lin[m];
    }
    cfg.dt = q.params.dt;
    cfg.qm = q.params.qm;
    cfg.alpha = q.params.alpha;
    cfg.pc_ref = q.params.pc_ref;
    cfg.tau_constants = q.params.tau_constants;
    cfg.sort_every = q.params.sort_every;
    cfg.mode = q.params.mode;
    cfg.cell = q.params.centring == SG_CELL_CENTRED;
    sg_particles hp;
    std::memset(&hp, 0, sizeof(hp));
    hp.n = q.particles.n;
    hp.on_device = 0;
    for (int m = 0; m < q.dim; ++m) {
      hp.u[m] = r->u[m].data();
      hp.v[m] = r->v[m].data();
    }
    hp.w = r->w.data();
    r->eng = make_engine(q.params.precision, q.dim);
    const int st = r->eng ? r->eng->init(cfg, &hp, r->stream) : SG_ERR_OOM;
    if (st != SG_OK) {
      const std::string keep = last_error();
      finish(s, r, SG_REQ_FAILED);
      set_error("admission of request " + std::to_string(r->ticket) + " failed: " + keep);
      *failed = st;
      continue;
    }
    r->state = SG_REQ_RUNNING;
    s->resident.push_back(r);
  }
  return SG_OK;
}

// One step of every resident run that still has steps to take: each run
// launches its own cached step graph (captured once per particle-buffer
// parity and sort phase) on its own stream, all forked from the server's
// stream and joined back, so the runs' kernels overlap on the device and
// no graph is captured again when the resident set changes.
// The job table of one precision to the device (on the server's stream;
// the pinned copy stays untouched until the tick's end synchronises).
static int stage_jobs(sg_server* s, int pi, const std::vector<unsigned char>& jobs) {
  const size_t bytes = jobs.size();
  if (bytes > s->jobs_cap[pi]) {
    if (s->jobs_dev[pi]) SG_CUDA(cudaFreeAsync(s->jobs_dev[pi], s->ds));
    if (s->jobs_host[pi]) cudaFreeHost(s->jobs_host[pi]);
    s->jobs_dev[pi] = s->jobs_host[pi] = nullptr;
    s->jobs_cap[pi] = 0;
    const size_t cap = bytes * 2;
    SG_CUDA(cudaMallocAsync(&s->jobs_dev[pi], cap, s->ds));
    SG_CUDA(cudaHostAlloc(&s->jobs_host[pi], cap, cudaHostAllocDefault));
    s->jobs_cap[pi] = cap;
  }
  std::memcpy(s->jobs_host[pi], jobs.data(), bytes);
  SG_CUDA(cudaMemcpyAsync(s->jobs_dev[pi], s->jobs_host[pi], bytes, cudaMemcpyHostToDevice, s->ds));
  return SG_OK;
}

// Batched tick.  Runs of the combination mode with a fixed tau, grids that
// fit one block and at most kCrossRunMaxParticles particles take their step
// in three parts: each run's graph up to its solve on its own stream; one
// launch per precision solving the component grids of all of them (one
// block per (run, grid)); each run's combination graph.  Other runs replay
// their whole step graph.  Every stream forks from the server's stream and
// joins it again.  The shared solve waits for the slowest run's particle
// stages, so larger runs, whose step is not bound by launch latency, keep
// their own solve.
constexpr size_t kCrossRunMaxParticles = (size_t)1 << 20;
static int tick_batched(sg_server* s, std::vector<Request*>& act) {
  SG_CUDA(cudaEventRecord(s->ev_start, s->ds));
  SG_CUDA(cudaEventRecord(s->fork, s->ds));
  std::vector<Request*> grp, rest;
  for (Request* r : act)
    (r->eng->solve_batchable() && r->eng->n_particles() <= kCrossRunMaxParticles ? grp : rest).push_back(r);
  for (Request* r : rest) {
    SG_CUDA(cudaStreamWaitEvent(r->stream, s->fork, 0));
    SG_TRY(r->eng->step(1));
    SG_CUDA(cudaEventRecord(r->ev1, r->stream));
  }
  std::vector<unsigned char> jobs[2];
  int max_size[2] = {0, 0}, max_log[2] = {0, 0};
  for (Request* r : grp) {
    SG_CUDA(cudaStreamWaitEvent(r->stream, s->fork, 0));
    SG_TRY(r->eng->step_pre());
    SG_CUDA(cudaEventRecord(r->ev0, r->stream));
    SG_CUDA(cudaStreamWaitEvent(s->ds, r->ev0, 0));
    const int pi = r->eng->real_bytes() == 8 ? 1 : 0;
    SG_TRY(r->eng->solve_jobs(jobs[pi], &max_size[pi], &max_log[pi]));
  }
  for (int pi = 0; pi < 2; ++pi) {
    if (jobs[pi].empty()) continue;
    SG_TRY(stage_jobs(s, pi, jobs[pi]));
    int nj;
    if (pi == 0) {
      nj = (int)(jobs[pi].size() / sizeof(SolveJob<float>));
      SG_TRY(launch_solve_batch<float>(static_cast<const SolveJob<float>*>(s->jobs_dev[pi]), nj, max_size[pi],
                                       max_log[pi], s->ds));
    } else {
      nj = (int)(jobs[pi].size() / sizeof(SolveJob<double>));
      SG_TRY(launch_solve_batch<double>(static_cast<const SolveJob<double>*>(s->jobs_dev[pi]), nj, max_size[pi],
                                        max_log[pi], s->ds));
    }
    ++s->solve_launches;
    s->solve_grids += (unsigned long long)nj;
  }
  SG_CUDA(cudaEventRecord(s->solved, s->ds));
  for (Request* r : grp) {
    SG_CUDA(cudaStreamWaitEvent(r->stream, s->solved, 0));
    SG_TRY(r->eng->step_post());
    SG_CUDA(cudaEventRecord(r->ev1, r->stream));
  }
  for (Request* r : act) SG_CUDA(cudaStreamWaitEvent(s->ds, r->ev1, 0));
  SG_CUDA(cudaEventRecord(s->ev_end, s->ds));
  SG_CUDA(cudaEventSynchronize(s->ev_end));
  float tick_ms = 0;
  SG_CUDA(cudaEventElapsedTime(&tick_ms, s->ev_start, s->ev_end));
  s->device_ms += tick_ms;
  for (Request* r : act) {
    float ms = 0;
    SG_CUDA(cudaEventElapsedTime(&ms, s->ev_start, r->ev1));
    s->step_ms.push_back(ms);
  }
  return SG_OK;
}

// Latency of a run's step is measured from the tick's start in both modes
// (a request advances one step per tick, whatever the other runs do).  The
// plain mode chains the runs on the device (each run's stream waits for the
// previous run's step) and synchronises once per tick, like the batched
// mode, so the two differ in launch structure only.
static int tick_plain(sg_server* s, std::vector<Request*>& act) {
  SG_CUDA(cudaEventRecord(s->ev_start, s->ds));
  cudaEvent_t last = s->ev_start;
  for (Request* r : act) {
    SG_CUDA(cudaStreamWaitEvent(r->stream, last, 0));
    SG_TRY(r->eng->step_plain());
    SG_CUDA(cudaEventRecord(r->ev1, r->stream));
    last = r->ev1;
  }
  SG_CUDA(cudaEventSynchronize(last));
  for (Request* r : act) {
    float ms = 0;
    SG_CUDA(cudaEventElapsedTime(&ms, s->ev_start, r->ev1));
    s->step_ms.push_back(ms);
  }
  float tick_ms = 0;
  SG_CUDA(cudaEventElapsedTime(&tick_ms, s->ev_start, last));
  s->device_ms += tick_ms;
  return SG_OK;
}

extern "C" {

int sg_serve_create(size_t hbm_budget_bytes, int max_slots, sg_server** out) {
  if (!out) return serr("sg_serve_create: out is NULL");
  if (max_slots < 1 || hbm_budget_bytes == 0) return serr("sg_serve_create: need max_slots >= 1 and a budget");
  sg_server* s = new sg_server;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  if (cudaStreamCreateWithFlags(&s->ds, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&s->ev_start) != cudaSuccess || cudaEventCreate(&s->ev_end) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->solved, cudaEventDisableTiming) != cudaSuccess) {
    delete s;
    return serr("sg_serve_create: stream/event creation failed", SG_ERR_CUDA);
  }
  *out = s;
  return SG_OK;
}

int sg_serve_set_mode(sg_server* s, int mode) {
  if (!s) return serr("sg_serve_set_mode: NULL server");
  if (mode != SG_SERVE_BATCHED && mode != SG_SERVE_PLAIN) return serr("sg_serve_set_mode: unknown mode");
  std::lock_guard<std::mutex> lk(s->mu);
  s->mode = mode;
  return SG_OK;
}

int sg_serve_submit(sg_server* s, const sg_request* req, unsigned long long* ticket) {
  if (!s || !req || !ticket) return serr("sg_serve_submit: NULL argument");
  const sg_particles& p = req->particles;
  if (p.on_device) return serr("sg_serve_submit: particle arrays must be host memory", SG_ERR_UNSUPPORTED);
  if (req->params.mode != SG_MODE_COMBINE && req->params.mode != SG_MODE_FILTER)
    return serr("sg_serve_submit: mode must be SG_MODE_COMBINE or SG_MODE_FILTER");
  if (req->params.centring != SG_NODE_CENTRED && req->params.centring != SG_CELL_CENTRED)
    return serr("sg_serve_submit: centring must be SG_NODE_CENTRED or SG_CELL_CENTRED");
  if (req->dim != 2 && req->dim != 3) return serr("sg_serve_submit: dim must be 2 or 3");
  if (req->nsteps < 0) return serr("sg_serve_submit: nsteps < 0");
  if (req->params.tau == SG_TAU_ADAPTIVE) return serr("sg_serve_submit: adaptive tau is not served", SG_ERR_UNSUPPORTED);
  int tau = req->params.tau;
  if (tau < 1 || tau > req->level_n || req->level_n < 2 || req->dim * req->level_n > 24)
    return serr("sg_serve_submit: bad level / tau");
  size_t rs = req->params.precision == SG_FP64 ? 8 : 4;
  Request* r = new Request;
  r->req = *req;
  for (int m = 0; m < req->dim; ++m) {
    if (p.n && (!p.u[m] || !p.v[m])) {
      delete r;
      return serr("sg_serve_submit: NULL particle array");
    }
    r->u[m].assign((const char*)p.u[m], (const char*)p.u[m] + p.n * rs);
    r->v[m].assign((const char*)p.v[m], (const char*)p.v[m] + p.n * rs);
  }
  if (p.n && !p.w) {
    delete r;
    return serr("sg_serve_submit: NULL charge array");
  }
  r->w.assign((const char*)p.w, (const char*)p.w + p.n * rs);
  r->footprint = estimate_footprint(req->params.precision, req->dim, req->level_n, tau, p.n);
  if (r->footprint > s->budget) {
    delete r;
    return serr("sg_serve_submit: request larger than the whole memory budget", SG_ERR_OOM);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  r->steps_left = req->nsteps;
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  return SG_OK;
}

int sg_serve_tick(sg_server* s, int* active) {
  if (!s) return serr("sg_serve_tick: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  bool changed = false;
  int admit_failed = SG_OK;
  SG_TRY(admit(s, &changed, &admit_failed));
  std::vector<Request*> act;
  for (Request* r : s->resident)
    if (r->steps_left > 0) act.push_back(r);
  int tick_status = SG_OK;
  if (!act.empty()) {
    int st = s->mode == SG_SERVE_BATCHED ? tick_batched(s, act) : tick_plain(s, act);
    if (st != SG_OK) {
      tick_status = st;  // the runs of this tick fail; the error is reported to the caller
      for (Request* r : act) r->steps_left = -1;
    } else {
      for (Request* r : act) {
        s->particle_steps += (double)r->req.particles.n;
        ++s->steps_served;
        --r->steps_left;
      }
    }
  }
  std::vector<Request*> keep;
  for (Request* r : s->resident) {
    if (r->steps_left == 0) {
      finish(s, r, SG_REQ_DONE);
      changed = true;
    } else if (r->steps_left < 0) {
      finish(s, r, SG_REQ_FAILED);
      changed = true;
    } else {
      keep.push_back(r);
    }
  }
  s->resident.swap(keep);
  (void)changed;
  if (active) *active = (int)s->resident.size();
  return tick_status != SG_OK ? tick_status : admit_failed;
}

int sg_serve_poll(sg_server* s, unsigned long long ticket, int* state, sg_diag* last) {
  if (!s || !state) return serr("sg_serve_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return serr("sg_serve_poll: unknown ticket");
  Request* r = it->second;
  *state = r->state;
  if (last) {
    if (r->state == SG_REQ_RUNNING && r->eng) r->eng->diagnostics(&r->last);
    *last = r->last;
  }
  return SG_OK;
}

int sg_serve_result(sg_server* s, unsigned long long ticket, const sg_particles_out* out) {
  if (!s || !out) return serr("sg_serve_result: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return serr("sg_serve_result: unknown ticket");
  Request* r = it->second;
  if (r->state != SG_REQ_DONE) return serr("sg_serve_result: request not finished", SG_ERR_STATE);
  if (out->n != r->req.particles.n) return serr("sg_serve_result: size mismatch", SG_ERR_SIZE);
  if (out->on_device) return serr("sg_serve_result: host buffers only", SG_ERR_UNSUPPORTED);
  size_t bytes = r->result_w.size();
  for (int m = 0; m < r->req.dim; ++m) {
    if (out->u[m]) std::memcpy(out->u[m], r->result_u[m].data(), bytes);
    if (out->v[m]) std::memcpy(out->v[m], r->result_v[m].data(), bytes);
  }
  if (out->w) std::memcpy(out->w, r->result_w.data(), bytes);
  return SG_OK;
}

int sg_serve_stats(sg_server* s, double* p50_ms, double* p99_ms, double* particle_steps_per_s,
                   unsigned long long* steps_served) {
  if (!s) return serr("sg_serve_stats: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->step_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
    return v[std::min(i, v.size() - 1)];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (particle_steps_per_s) *particle_steps_per_s = s->device_ms > 0 ? s->particle_steps / (s->device_ms * 1e-3) : 0.0;
  if (steps_served) *steps_served = s->steps_served;
  return SG_OK;
}

int sg_serve_solve_stats(sg_server* s, unsigned long long* launches, unsigned long long* grids) {
  if (!s) return serr("sg_serve_solve_stats: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (launches) *launches = s->solve_launches;
  if (grids) *grids = s->solve_grids;
  return SG_OK;
}

void sg_serve_destroy(sg_server* s) {
  if (!s) return;
  for (Request* r : s->resident) finish(s, r, SG_REQ_FAILED);
  for (auto& kv : s->all) delete kv.second;
  for (int pi = 0; pi < 2; ++pi) {
    if (s->jobs_dev[pi]) cudaFreeAsync(s->jobs_dev[pi], s->ds);
    if (s->jobs_host[pi]) cudaFreeHost(s->jobs_host[pi]);
  }
  if (s->ds) cudaStreamSynchronize(s->ds);
  if (s->ev_start) cudaEventDestroy(s->ev_start);
  if (s->ev_end) cudaEventDestroy(s->ev_end);
  if (s->fork) cudaEventDestroy(s->fork);
  if (s->solved) cudaEventDestroy(s->solved);
  if (s->ds) cudaStreamDestroy(s->ds);
  delete s;
}

}  // extern "C"
