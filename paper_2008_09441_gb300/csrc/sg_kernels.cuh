// Launchers of the library's device kernels (host side).  Every launcher
// enqueues on the given stream and returns an SG_* status.
#pragma once

#include <cmath>
#include <vector>

#include "sg_common.cuh"

namespace sg {

// ---------------------------------------------------------------- sort
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // keys per tile

struct SortScratch {
  uint32_t* tile_hist = nullptr;   // 256 * ntiles
  uint32_t* block_sums = nullptr;  // scan block totals
  size_t ntiles = 0;
};

size_t sort_scratch_words(size_t np);  // u32 words needed for SortScratch
void sort_scratch_bind(SortScratch& s, uint32_t* base, size_t np);

// keys[i] = Morton key of particle i's level-n cell, idx[i] = i,
// *checksum += sum_i (keys[i] + 1).
template <typename real, int D>
int launch_keys(const PArrays<real, D>& p, size_t np, int n, uint32_t* keys, uint32_t* idx,
                unsigned long long* checksum, unsigned* status, cudaStream_t s);

// Same for positions given as plain arrays (stand-alone sort entry point).
template <typename real, int D>
int launch_keys_raw(const real* const* u, size_t np, int n, uint32_t* keys, uint32_t* idx,
                    unsigned long long* checksum, unsigned* status, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// Ping-pongs between (keys, vals) and (keys_alt, vals_alt); *in_alt tells
// where the sorted result ended.  If vals_identity, the first pass uses the
// input index as value instead of reading vals.
int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                     size_t np, int bits, bool vals_identity, SortScratch& scr, cudaStream_t s,
                     bool* in_alt);

template <typename real, int D>
int launch_permute(const PArrays<real, D>& src, const PArrays<real, D>& dst, const uint32_t* perm,
                   size_t np, cudaStream_t s);

// dst[pid[i]] = src[i] for every particle array (back to the original order).
template <typename real, int D>
int launch_unpermute(const PArrays<real, D>& src, const PArrays<real, D>& dst, size_t np, cudaStream_t s);

// counts[key] += 1 for every sorted key (counts zeroed by the caller).
int launch_counts(const uint32_t* keys, size_t np, uint32_t* counts, cudaStream_t s);

// Exclusive scan of m u32 values (out may equal in).
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, size_t m, uint32_t* block_sums,
                       cudaStream_t s);
size_t scan_block_sums_words(size_t m);

// ---------------------------------------------------------------- deposit
constexpr int DEP_THREADS = 512;
constexpr int DEP_ITEMS = 4;
constexpr int DEP_CHUNK = DEP_THREADS * DEP_ITEMS;

// scale / inv_scale: the FP32 fixed-point scale of the window (WinAcc), 1 for FP64.
// shift: position of node 0 in cells (0 node-centred, 1/2 cell-centred).
template <typename real, int D>
int launch_deposit(const PArrays<real, D>& p, size_t np, int n, real inv_cell_vol, real* rho,
                   int win_cap_nodes, real scale, real inv_scale, real shift, cudaStream_t s);

// The upload's statistics, out[0 .. 2 nb]: per-block FP64 charge sums, per-
// block max |q|, then the status word (its bits in a double).
template <typename real>
int launch_charge_stats(const real* w, size_t n, const unsigned* status, double* out, int nblocks, cudaStream_t s);


// ---------------------------------------------------------------- line passes
// The lines of one array along one axis, processed by one kernel launch
// together with the other jobs of the same pass.
constexpr int RJ_LEVELS = 13;  // levels 0..12 (2D n <= 12, 3D n <= 8)
struct LineJob {
  const void* src;       // [outer][2^top][inner] reals
  int top;               // log2 of the line length
  int outer, inner;      // powers of two; lines = outer * inner
  int block_begin;       // first block of this job in the launch
  int tile_stride;       // reals per tile row in shared memory (inner > 1)
  int tmask;             // bit l set: level l is written
  int tmin;              // lowest level written
  int sub_mean;          // 1: the source is the regular grid; the mean is subtracted as it is read
  void* dst[RJ_LEVELS];  // level l: [outer][2^l][inner]
};

// Block -> job of a pass: the last job whose block_begin <= blockIdx.x.  The
// first warp reads 32 job headers at a time (no chain of dependent loads).
template <typename Job>
__device__ __forceinline__ int find_job(const Job* __restrict__ jobs, int njobs) {
  __shared__ int s_job;
  const int b = blockIdx.x;
  if (threadIdx.x < 32) {
    int best = 0;
    for (int base = 0; base < njobs; base += 32) {
      const int idx = base + (int)threadIdx.x;
      const bool le = idx < njobs && jobs[idx].block_begin <= b;
      const unsigned m = __ballot_sync(0xffffffffu, le);
      if (m) best = base + 31 - __clz(m);
      if (m != 0xffffffffu) break;
    }
    if (threadIdx.x == 0) s_job = best;
  }
  __syncthreads();
  return s_job;
}

// Restriction along one axis of every job's lines (full weighting 1/4,
// 1/2, 1/4 per level halving, the exact form of R along one axis for nested
// node-centred grids; cell = true: R of cell-centred grids through the
// face-averaged cascade), outputs in the natural layout.  Jobs that read
// the regular grid subtract `mean` (Q / |box|) from every value they read:
// the component densities are stored as deviations from the mean, which
// every R_i preserves (its weights sum to one), so that FP32 rounding in the
// restriction sums, in storage and in the transforms is relative to the
// density's fluctuation instead of its much larger uniform part.
template <typename real>
int launch_restrict_pass(const LineJob* jobs_dev, int njobs, int nblocks, int lines_per_block, int vpl,
                         int smem_bytes, bool cell, real mean, cudaStream_t s);

// FFT passes over the component grids.
enum FftKind { FFT_FWD_FIRST = 0, FFT_FWD_MID = 1, FFT_LAST = 2, FFT_INV_MID = 3, FFT_INV_LAST = 4 };

struct FftJob {
  int grid;          // index into the grid table
  int dims[3];
  int axis;
  int logn;
  int lines;
  int lines_per_block;
  int block_begin;
  int comp;          // inverse passes: component pair (2 comp, 2 comp + 1)
};

// FFT twiddles, stage-major: the butterflies of span 2h (h = 1, 2, 4, ...)
// use W_{2h}^p = exp(-2 pi i p / (2h)) for p < h, stored at h - 1 + p, so
// that consecutive butterflies of a stage read consecutive entries.  A table
// for transforms of up to 2^L points holds 2^L - 1 entries.
__host__ __device__ constexpr int twiddle_index(int h, int p) { return h - 1 + p; }
__host__ __device__ constexpr int twiddle_count(int L) { return L < 1 ? 1 : (1 << L) - 1; }
template <typename real>
std::vector<cplx<real>> make_twiddles(int L) {
  std::vector<cplx<real>> tw((size_t)twiddle_count(L));
  tw[0] = {(real)1, (real)0};
  for (int h = 1; h < (1 << L); h <<= 1)
    for (int p = 0; p < h; ++p) {
      const double a = M_PI * (double)p / (double)h;
      tw[(size_t)twiddle_index(h, p)] = {(real)std::cos(a), (real)(-std::sin(a))};
    }
  return tw;
}

template <typename real>
struct SolveArena {
  const GridDesc* grids;
  const real* rho;     // S
  cplx<real>* A;       // S
  cplx<real>* B;       // D * S
  real* E;             // D * S
  size_t S;
  const cplx<real>* tw;  // make_twiddles(log_nmax)
  int log_nmax;
  int dim;
};

// Complex values per block of a transform pass (whole lines, at least one
// line per block); the block has half as many threads.
constexpr int FFT_BLOCK_VALUES = 1024;

template <typename real>
int launch_fft_pass(int kind, const SolveArena<real>& a, const FftJob* jobs_dev, int njobs,
                    int nblocks, int smem_bytes, cudaStream_t s);

// All component grids in one launch, one block per grid, whole grid in shared
// memory (used when every grid has at most SMALL_SOLVE_MAX<real> points).
template <typename real>
int launch_solve_small(const SolveArena<real>& a, int ngrids, int max_size, cudaStream_t s, int grid0 = 0);
template <typename real>
constexpr int small_solve_max() { return sizeof(real) == 4 ? 4096 : 2048; }

// One component grid of one run for the cross-run solve: the run's arena
// and the grid's index in it.  A launch over a table of these solves the
// component grids of every run in it, one block per (run, grid).
template <typename real>
struct SolveJob {
  SolveArena<real> a;
  int grid;
  int pad;
};
// max_size: largest grid of the table (points); max_log: largest log_nmax.
template <typename real>
int launch_solve_batch(const SolveJob<real>* jobs, int njobs, int max_size, int max_log, cudaStream_t s);

// The filter mode's regular-grid solve: rho_f -> E on the regular nodes
// (E_hi node-interleaved with `stride`, FP32 low planes zeroed), per-block
// field-energy partials at partials[pair * blocks + block] (ceil(dim/2) pairs).
// rho_f is the combination of the component densities, a deviation from the
// mean like them.
template <typename real>
int launch_regular_solve(const real* rho_f, cplx<real>* A, cplx<real>* B, const real* ktab,
                         const cplx<real>* tw, int dim, int n, real* Ehi, float* Elo, int stride, double* partials,
                         int blocks, cudaStream_t s);

// Generic in-place complex FFT of a whole N^D array (regular grid) along one
// axis, forward or inverse (unnormalised), in the given precision.
template <typename real>
int launch_fft_array_axis(cplx<real>* data, int D, int logn, int axis, bool inverse,
                          const cplx<real>* tw, int log_nmax, cudaStream_t s);

// ---------------------------------------------------------------- combine
// Grids grouped by their x level: grid[start[l] .. start[l+1]) have l_1 = l;
// start[l] for l > n holds the total count.
constexpr int CB_MAX_GRIDS = 128;
struct LevelLists {
  int start[18];
  const int* grid;
};



// ---------------------------------------------------------------- push
// The combined field the push gathers from is stored node-interleaved:
// E_hi[node * ec_stride<D>() + m] (2D: (E_x, E_y); 3D: (E_x, E_y, E_z, pad)),
// so one corner of the gather is one 8- or 16-byte load.  The low parts of
// the FP32 path's float pairs are planes E_lo[m * N_c + node].
template <int D>
constexpr int ec_stride() { return D == 2 ? 2 : 4; }

template <typename real>
struct PushParams {
  real qm, dt;
  real ke_fac;    // 1 / (2 q/m): kinetic energy 0.5 m_p v.v with m_p = q_p / (q/m)
  real dt_over_L[3];
  real eext[3];   // E_ext,m = eext[m] * (u_m - 1/2)   (eext = Eext_lin * L)
  real tB[3];     // q/m * B * dt / 2 (Boris t vector)
  int boris;
  int has_eext;
  int drift;      // 0: velocity only (initial half kick), 1: kick + drift
  real shift;     // position of node 0 in cells: 0 node-centred, 1/2 cell-centred
};

// Sort work fused into the push on sort steps (keys == nullptr: none).
struct SortFuse {
  uint32_t* keys = nullptr;        // tile key per particle (storage order)
  unsigned long long* checksum = nullptr;
  int tile_shift = 0;              // tile = level-n Morton key >> (D * tile_shift)
};

template <typename real, int D>
int launch_push(const PArrays<real, D>& p, size_t np, int n, const real* Ecomb, PushParams<real> pp,
                double* ke_partials, unsigned* status, const SortFuse& sf, cudaStream_t s, int blocks = 0);
template <typename real, int D>
int push_blocks(size_t np);  // grid of the push (size of its kinetic-energy partials)

// ---------------------------------------------------------------- step sort (tile counting sort)
// Tile keys and counts of the current positions (the push emits them on sort
// steps; this kernel serves init and checkpoint load).
template <typename real, int D>
int launch_tile_keys(const PArrays<real, D>& p, size_t np, int n, const SortFuse& sf, unsigned* status,
                     cudaStream_t s);
// tile_count[key] += 1 for every key (counts zeroed by the caller).
int launch_tile_hist(const uint32_t* keys, size_t np, uint32_t* tile_count, cudaStream_t s);
// Scatter every particle to its tile's next free slot (cursor = exclusive
// scan of the tile counts): one pass, reads key + payload, writes payload.
template <typename real, int D>
int launch_tile_scatter(const PArrays<real, D>& src, const PArrays<real, D>& dst, const uint32_t* keys,
                        uint32_t* cursor, size_t np, cudaStream_t s);

// ---------------------------------------------------------------- misc
template <typename real, int D>
int launch_wrap_check(const PArrays<real, D>& p, size_t np, unsigned* status, cudaStream_t s);


// Device diagnostics record updated at the end of each step.
struct DevDiag {
  double field_energy;
  double field_energy_prev;
  double kinetic_energy;
  unsigned long long checksum;
  unsigned status;
  unsigned pad;
};

int launch_finalize_step(const double* fe_partials, int n_fe, const double* ke_partials, int n_ke,
                         double fe_scale, DevDiag* dd, cudaStream_t s);

// The diagnostics record in one buffer, for one device-to-host copy: *dd at
// 0, *cks at o_cks, *st at o_cks + 8, and V_i sum_k rho_i(x_k) of every grid
// (FP64) from o_ch on (one block per grid).
template <typename real>
int launch_diag_record(const GridDesc* grids, int ngrids, const real* rho, const DevDiag* dd,
                       const unsigned long long* cks, const unsigned* st, void* out, size_t o_cks, size_t o_ch,
                       cudaStream_t s);

// Step bookkeeping closed by the last block of the combination kernel:
// field energy from the per-row partials (scaled by fe_scale), the previous
// field energy, and the kinetic energy from the push partials when given.
struct CombineFinal {
  int active;
  int n_ke;
  const double* ke_partials;
  double fe_scale;
  DevDiag* dd;
  unsigned* counter;  // zero between launches; the last block resets it
};

template <typename real, int D>
int launch_combine(const GridDesc* grids, const LevelLists& ll, int lmin, const real* E, size_t S, int n,
                   real* Ehi, float* Elo, double* energy_partials, const CombineFinal& fin,
                   cudaStream_t s, int ncomp,  // ncomp = D: the fields, interleaved; 1: a density, plain
                   bool cell,                  // cell-centred grids
                   bool fp64_acc);             // FP32 path: accumulate in double instead of float-float

template <typename real>
int launch_to_double(const real* src, double* dst, size_t n, cudaStream_t s);
// dst[m * nd + node] = E_hi[node * stride + m] (+ E_lo[m * nd + node] when lo != nullptr), FP64.
template <typename real>
int launch_field_to_double(const real* hi, const float* lo, double* dst, size_t nd, int dim, int stride,
                           cudaStream_t s);

// ---------------------------------------------------------------- tau estimator
int launch_real_to_cplx(const double* src, cplx<double>* dst, size_t n, double scale, cudaStream_t s);
int launch_maxabs_cplx(const cplx<double>* z, size_t n, double* out_max, cudaStream_t s);
int launch_maxabs_real_part(const cplx<double>* z, size_t n, double* out_max, cudaStream_t s);
int launch_maxabs_real(const double* x, size_t n, double* out_max, cudaStream_t s);
int launch_threshold(cplx<double>* z, size_t n, const double* maxabs, double frac, cudaStream_t s);
int launch_kmult(const cplx<double>* src, cplx<double>* dst, int D, int logn, const double* kfac,
                 int mask, cudaStream_t s);
int launch_maxabs_kmult(const cplx<double>* src, int D, int logn, const double* kfac, int mask,
                        double* out_max, cudaStream_t s);

}  // namespace sg
