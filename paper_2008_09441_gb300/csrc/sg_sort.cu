// Cell-key sort of the particles: Morton keys of the level-n cells, a stable
// LSD radix sort of (key, index) pairs with 8-bit digits, the permutation of
// the particle arrays and per-cell counts.  Integer work, bit-exact.
#include "sg_kernels.cuh"

namespace sg {


// ---------------------------------------------------------------- keys
template <typename real, int D>
__global__ void __launch_bounds__(256) k_keys(PArrays<real, D> p, size_t np, int n, uint32_t* keys,
                                              uint32_t* idx, unsigned long long* checksum,
                                              unsigned* status) {
  const int N = 1 << n;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long part = 0;
  if (i < np) {
    int c[D];
    bool bad = false;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      real u = p.u[m][i];
      bad |= !(u >= (real)0 && u < (real)1);
      c[m] = cell_of(u, n, N);
    }
    if (bad) atomicOr(status, ST_KEY_RANGE);
    uint32_t k = morton_key<D>(c, n);
    keys[i] = k;
    if (idx) idx[i] = (uint32_t)i;
    part = (unsigned long long)k + 1ull;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0 && checksum && part) atomicAdd(checksum, part);
}

template <typename real, int D>
struct RawU {
  const real* u[D];
};

template <typename real, int D>
__global__ void __launch_bounds__(256) k_keys_raw(RawU<real, D> r, size_t np, int n, uint32_t* keys,
                                                  uint32_t* idx, unsigned long long* checksum,
                                                  unsigned* status) {
  const int N = 1 << n;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long part = 0;
  if (i < np) {
    int c[D];
    bool bad = false;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      real u = r.u[m][i];
      bad |= !(u >= (real)0 && u < (real)1);
      // positions outside [0,1) are wrapped first (periodic box)
      if (bad) u = wrap_unit(u);
      c[m] = cell_of(u, n, N);
    }
    uint32_t k = morton_key<D>(c, n);
    keys[i] = k;
    if (idx) idx[i] = (uint32_t)i;
    part = (unsigned long long)k + 1ull;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0 && checksum && part) atomicAdd(checksum, part);
}

template <typename real, int D>
int launch_keys(const PArrays<real, D>& p, size_t np, int n, uint32_t* keys, uint32_t* idx,
                unsigned long long* checksum, unsigned* status, cudaStream_t s) {
  if (np == 0) return SG_OK;
  k_keys<real, D><<<(unsigned)((np + 255) / 256), 256, 0, s>>>(p, np, n, keys, idx, checksum, status);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template <typename real, int D>
int launch_keys_raw(const real* const* u, size_t np, int n, uint32_t* keys, uint32_t* idx,
                    unsigned long long* checksum, unsigned* status, cudaStream_t s) {
  if (np == 0) return SG_OK;
  RawU<real, D> r;
  for (int m = 0; m < D; ++m) r.u[m] = u[m];
  k_keys_raw<real, D><<<(unsigned)((np + 255) / 256), 256, 0, s>>>(r, np, n, keys, idx, checksum, status);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// ---------------------------------------------------------------- scan
constexpr int SC_THREADS = 1024;  // short serial runs per thread: the scan is latency-bound
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

size_t scan_block_sums_words(size_t m) { return (m + SC_TILE - 1) / SC_TILE + 1; }

// Block-wide exclusive scan of SC_TILE values staged in shared memory.
__device__ void block_exclusive_scan_tile(uint32_t* sh, uint32_t* total) {
  __shared__ uint32_t warp_tot[SC_THREADS / 32];
  int t = threadIdx.x;
  uint32_t loc[SC_ITEMS];
  uint32_t run = 0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    loc[j] = run;
    run += sh[t * SC_ITEMS + j];
  }
  // inclusive warp scan of per-thread totals
  uint32_t x = run;
  int lane = t & 31, w = t >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t v = lane < SC_THREADS / 32 ? warp_tot[lane] : 0;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < SC_THREADS / 32) warp_tot[lane] = inc - v;  // exclusive
    if (lane == SC_THREADS / 32 - 1) *total = inc;
  }
  __syncthreads();
  uint32_t base = warp_tot[w] + (x - run);
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) sh[t * SC_ITEMS + j] = base + loc[j];
  __syncthreads();
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_tiles(const uint32_t* in, uint32_t* out, size_t m,
                                                           uint32_t* block_sums) {
  __shared__ uint32_t sh[SC_TILE];
  __shared__ uint32_t tot;
  size_t base = (size_t)blockIdx.x * SC_TILE;
  for (int j = threadIdx.x; j < SC_TILE; j += SC_THREADS) sh[j] = (base + j < m) ? in[base + j] : 0u;
  __syncthreads();
  block_exclusive_scan_tile(sh, &tot);
  for (int j = threadIdx.x; j < SC_TILE; j += SC_THREADS)
    if (base + j < m) out[base + j] = sh[j];
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Exclusive scan of up to SC_TILE block sums in one block (repeated tiles if more).
__global__ void __launch_bounds__(SC_THREADS) k_scan_top(uint32_t* block_sums, int nb) {
  __shared__ uint32_t sh[SC_TILE];
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += SC_TILE) {
    for (int j = threadIdx.x; j < SC_TILE; j += SC_THREADS) sh[j] = (base + j < nb) ? block_sums[base + j] : 0u;
    __syncthreads();
    block_exclusive_scan_tile(sh, &tot);
    for (int j = threadIdx.x; j < SC_TILE; j += SC_THREADS)
      if (base + j < nb) block_sums[base + j] = sh[j] + carry;
    __syncthreads();
    carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_add(uint32_t* out, size_t m, const uint32_t* block_sums) {
  size_t base = (size_t)blockIdx.x * SC_TILE;
  uint32_t add = block_sums[blockIdx.x];
  if (add == 0) return;
  for (int j = threadIdx.x; j < SC_TILE; j += SC_THREADS)
    if (base + j < m) out[base + j] += add;
}

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, size_t m, uint32_t* block_sums, cudaStream_t s) {
  if (m == 0) return SG_OK;
  unsigned nb = (unsigned)((m + SC_TILE - 1) / SC_TILE);
  k_scan_tiles<<<nb, SC_THREADS, 0, s>>>(in, out, m, block_sums);
  SG_CHECK_LAUNCH();
  if (nb > 1) {
    k_scan_top<<<1, SC_THREADS, 0, s>>>(block_sums, (int)nb);
    SG_CHECK_LAUNCH();
    k_scan_add<<<nb, SC_THREADS, 0, s>>>(out, m, block_sums);
    SG_CHECK_LAUNCH();
  }
  return SG_OK;
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_WARP_KEYS = RS_TILE / RS_WARPS;
static_assert(RS_WARP_KEYS == 32 * RS_ITEMS, "one key per lane per chunk");

size_t sort_scratch_words(size_t np) {
  size_t ntiles = (np + RS_TILE - 1) / RS_TILE;
  if (ntiles == 0) ntiles = 1;
  return 256 * ntiles + scan_block_sums_words(256 * ntiles) + 64;
}

void sort_scratch_bind(SortScratch& s, uint32_t* base, size_t np) {
  size_t ntiles = (np + RS_TILE - 1) / RS_TILE;
  if (ntiles == 0) ntiles = 1;
  s.ntiles = ntiles;
  s.tile_hist = base;
  s.block_sums = base + 256 * ntiles;
}

// Digit histogram of one tile; keys with equal digits in a warp are counted
// by their leader (match_any aggregation) to avoid shared atomic pile-ups on
// nearly sorted input.
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t* keys, size_t n, int shift,
                                                           uint32_t* hist, int ntiles) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += RS_THREADS) h[i] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * RS_TILE;
  int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    size_t idx = base + i;
    bool valid = idx < n;
    uint32_t dg = valid ? ((keys[idx] >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, dg);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[dg], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += RS_THREADS) hist[(size_t)i * ntiles + blockIdx.x] = h[i];
}

// Stable scatter of one tile: warp w owns keys [w*512, (w+1)*512) of the
// tile, taken in 16 chunks of 32 in order; the rank of a key is the count
// of earlier equal digits in its warp segment, then the warp-ordered prefix,
// then the tile's global offset for the digit.
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint32_t* keys_in, const uint32_t* vals_in,
                                                              size_t n, int shift, const uint32_t* offsets,
                                                              int ntiles, uint32_t* keys_out,
                                                              uint32_t* vals_out, int vals_identity) {
  __shared__ uint32_t wh[RS_WARPS][256];
  __shared__ uint32_t tile_off[256];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wh[0][0])[i] = 0;
  for (int i = threadIdx.x; i < 256; i += RS_THREADS) tile_off[i] = offsets[(size_t)i * ntiles + blockIdx.x];
  __syncthreads();
  size_t base = (size_t)blockIdx.x * RS_TILE + (size_t)w * RS_WARP_KEYS;
  uint32_t kk[RS_ITEMS], rank[RS_ITEMS];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int c = 0; c < RS_ITEMS; ++c) {
    size_t idx = base + (size_t)c * 32 + lane;
    bool valid = idx < n;
    uint32_t key = valid ? keys_in[idx] : 0u;
    uint32_t dg = valid ? ((key >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, dg);
    uint32_t before = valid ? wh[w][dg] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wh[w][dg] = before + (uint32_t)__popc(peers);
    __syncwarp();
    rank[c] = before + (uint32_t)__popc(peers & lt);
    kk[c] = key;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      uint32_t t = wh[ww][d];
      wh[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < RS_ITEMS; ++c) {
    size_t idx = base + (size_t)c * 32 + lane;
    if (idx < n) {
      uint32_t dg = (kk[c] >> shift) & 255u;
      uint32_t pos = tile_off[dg] + wh[w][dg] + rank[c];
      keys_out[pos] = kk[c];
      vals_out[pos] = vals_identity ? (uint32_t)idx : vals_in[idx];
    }
  }
}

int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, size_t np,
                     int bits, bool vals_identity, SortScratch& scr, cudaStream_t s, bool* in_alt) {
  *in_alt = false;
  if (np == 0) return SG_OK;
  if (np > 0xFFFFFFFFull) {
    set_error("radix sort: more than 2^32-1 particles");
    return SG_ERR_SIZE;
  }
  int ntiles = (int)((np + RS_TILE - 1) / RS_TILE);
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  int passes = (bits + 7) / 8;
  if (passes == 0) passes = 1;
  bool ident = vals_identity;
  for (int pass = 0; pass < passes; ++pass) {
    int shift = pass * 8;
    k_radix_hist<<<ntiles, RS_THREADS, 0, s>>>(ki, np, shift, scr.tile_hist, ntiles);
    SG_CHECK_LAUNCH();
    SG_TRY(exclusive_scan_u32(scr.tile_hist, scr.tile_hist, (size_t)256 * ntiles, scr.block_sums, s));
    k_radix_scatter<<<ntiles, RS_THREADS, 0, s>>>(ki, vi, np, shift, scr.tile_hist, ntiles, ko, vo, ident ? 1 : 0);
    SG_CHECK_LAUNCH();
    ident = false;
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    *in_alt = !*in_alt;
  }
  return SG_OK;
}

// ---------------------------------------------------------------- permute / counts
template <typename real, int D>
__global__ void __launch_bounds__(256) k_permute(PArrays<real, D> src, PArrays<real, D> dst, const uint32_t* perm,
                                                 size_t np) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  uint32_t j = perm[i];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    dst.u[m][i] = src.u[m][j];
    dst.v[m][i] = src.v[m][j];
  }
  dst.w[i] = src.w[j];
  dst.pid[i] = src.pid[j];
}

template <typename real, int D>
int launch_permute(const PArrays<real, D>& src, const PArrays<real, D>& dst, const uint32_t* perm, size_t np,
                   cudaStream_t s) {
  if (np == 0) return SG_OK;
  k_permute<real, D><<<(unsigned)((np + 255) / 256), 256, 0, s>>>(src, dst, perm, np);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template <typename real, int D>
__global__ void __launch_bounds__(256) k_unpermute(PArrays<real, D> src, PArrays<real, D> dst, size_t np) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  uint32_t j = src.pid[i];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    dst.u[m][j] = src.u[m][i];
    dst.v[m][j] = src.v[m][i];
  }
  dst.w[j] = src.w[i];
  if (dst.pid) dst.pid[j] = j;
}

template <typename real, int D>
int launch_unpermute(const PArrays<real, D>& src, const PArrays<real, D>& dst, size_t np, cudaStream_t s) {
  if (np == 0) return SG_OK;
  k_unpermute<real, D><<<(unsigned)((np + 255) / 256), 256, 0, s>>>(src, dst, np);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// ---------------------------------------------------------------- tile counting sort
// Tile keys of the current positions (the push emits them on sort steps;
// this kernel serves init and checkpoint load) and sum (cell key + 1).
template <typename real, int D>
__global__ void __launch_bounds__(256) k_tile_keys(PArrays<real, D> p, size_t np, int n, SortFuse sf,
                                                   unsigned* status) {
  const int N = 1 << n;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long part = 0;
  if (i < np) {
    int c[D];
    bool bad = false;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      real u = p.u[m][i];
      bad |= !(u >= (real)0 && u < (real)1);
      c[m] = cell_of(u, n, N);
    }
    if (bad) atomicOr(status, ST_KEY_RANGE);
    uint32_t k = morton_key<D>(c, n);
    sf.keys[i] = k >> (D * sf.tile_shift);
    part = (unsigned long long)k + 1ull;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0 && part && sf.checksum) atomicAdd(sf.checksum, part);
}

template <typename real, int D>
int launch_tile_keys(const PArrays<real, D>& p, size_t np, int n, const SortFuse& sf, unsigned* status,
                     cudaStream_t s) {
  if (np == 0) return SG_OK;
  k_tile_keys<real, D><<<(unsigned)((np + 255) / 256), 256, 0, s>>>(p, np, n, sf, status);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// Block-level counting.  A block takes TB_ITEMS consecutive keys (the
// particles were tile-sorted one step earlier, so the block sees a narrow
// range of tiles); when that range fits TB_SPAN shared counters the block
// counts there with native 32-bit shared atomics and issues one global
// atomic per distinct tile, otherwise each key adds to the global counter.
constexpr int TB_THREADS = 256;
constexpr int TB_PER_THREAD = 4;
constexpr int TB_ITEMS = TB_THREADS * TB_PER_THREAD;
constexpr int TB_SPAN = 1024;

__device__ __forceinline__ void block_key_range(const uint32_t (&t)[TB_PER_THREAD], uint32_t* s_lo, uint32_t* s_hi) {
  uint32_t lo = 0xFFFFFFFFu, hi = 0;
#pragma unroll
  for (int k = 0; k < TB_PER_THREAD; ++k)
    if (t[k] != 0xFFFFFFFFu) {
      lo = min(lo, t[k]);
      hi = max(hi, t[k]);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(s_lo, lo);
    atomicMax(s_hi, hi);
  }
}

// Keys of item k of thread t: chunk + k * TB_THREADS + t (coalesced rounds).
__device__ __forceinline__ void load_keys(const uint32_t* __restrict__ keys, size_t np, size_t chunk,
                                          uint32_t (&t)[TB_PER_THREAD]) {
#pragma unroll
  for (int k = 0; k < TB_PER_THREAD; ++k) {
    const size_t i = chunk + (size_t)k * TB_THREADS + threadIdx.x;
    t[k] = i < np ? __ldg(keys + i) : 0xFFFFFFFFu;
  }
}

__global__ void __launch_bounds__(TB_THREADS) k_tile_hist(const uint32_t* __restrict__ keys, size_t np,
                                                          uint32_t* tile_count) {
  __shared__ uint32_t s_cnt[TB_SPAN];
  __shared__ uint32_t s_lo, s_hi;
  const size_t chunk = (size_t)blockIdx.x * TB_ITEMS;
  uint32_t t[TB_PER_THREAD];
  load_keys(keys, np, chunk, t);
  if (threadIdx.x == 0) {
    s_lo = 0xFFFFFFFFu;
    s_hi = 0;
  }
  for (int i = threadIdx.x; i < TB_SPAN; i += TB_THREADS) s_cnt[i] = 0;
  __syncthreads();
  block_key_range(t, &s_lo, &s_hi);
  __syncthreads();
  const uint32_t lo = s_lo;
  const bool local = s_hi - lo < (uint32_t)TB_SPAN;
  const int lane = threadIdx.x & 31;
  // lanes with equal keys (the common case: sorted input) add once per group
#pragma unroll
  for (int k = 0; k < TB_PER_THREAD; ++k) {
    const unsigned peers = __match_any_sync(0xffffffffu, t[k]);
    if (t[k] == 0xFFFFFFFFu || lane != __ffs(peers) - 1) continue;
    if (local)
      atomicAdd(&s_cnt[t[k] - lo], (uint32_t)__popc(peers));
    else
      atomicAdd(&tile_count[t[k]], (uint32_t)__popc(peers));
  }
  if (!local) return;
  __syncthreads();
  for (int i = threadIdx.x; i < TB_SPAN; i += TB_THREADS)
    if (s_cnt[i]) atomicAdd(&tile_count[lo + i], s_cnt[i]);
}

int launch_tile_hist(const uint32_t* keys, size_t np, uint32_t* tile_count, cudaStream_t s) {
  if (np == 0) return SG_OK;
  k_tile_hist<<<(unsigned)((np + TB_ITEMS - 1) / TB_ITEMS), TB_THREADS, 0, s>>>(keys, np, tile_count);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// Scatter every particle to its tile's slots.  Same blocks as the count.
// When the block's keys span at most TB_SPAN tiles (the usual case: the
// particles were tile-sorted a few steps earlier), the block ranks its
// particles per tile with shared atomics, reserves one range per distinct
// tile with a single global atomic, orders its payload by tile in shared
// memory (a block-local counting sort), and writes it out as contiguous runs
// per tile -- coalesced stores even when the particles have drifted over
// many tiles.  Wider blocks reserve per warp group and store directly.
// Within a tile the order depends on the atomics: the step sort is a valid,
// not a stable, counting sort by tile key.
template <typename real, int D>
struct ScatterStage {
  static constexpr size_t bytes = (size_t)TB_ITEMS * ((2 * D + 1) * sizeof(real) + 2 * sizeof(uint32_t));
  static constexpr bool on = bytes <= 160 * 1024;
};

template <typename real, int D>
__global__ void __launch_bounds__(TB_THREADS) k_tile_scatter(PArrays<real, D> src, PArrays<real, D> dst,
                                                             const uint32_t* __restrict__ keys, uint32_t* cursor,
                                                             size_t np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_cnt[TB_SPAN];   // per tile: count, then the local start
  __shared__ uint32_t s_base[TB_SPAN];  // per tile: the block's global base
  __shared__ uint32_t s_wsum[TB_THREADS / 32];
  __shared__ uint32_t s_lo, s_hi;
  const size_t chunk = (size_t)blockIdx.x * TB_ITEMS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t t[TB_PER_THREAD];
  load_keys(keys, np, chunk, t);
  // the payload's loads go out now, so that their latency overlaps the ranking
  real pu[TB_PER_THREAD][D], pv[TB_PER_THREAD][D], pw[TB_PER_THREAD];
  uint32_t ppid[TB_PER_THREAD];
#pragma unroll
  for (int k = 0; k < TB_PER_THREAD; ++k) {
    const size_t i = chunk + (size_t)k * TB_THREADS + threadIdx.x;
    const bool valid = i < np;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      pu[k][m] = valid ? __ldg(src.u[m] + i) : (real)0;
      pv[k][m] = valid ? __ldg(src.v[m] + i) : (real)0;
    }
    pw[k] = valid ? __ldg(src.w + i) : (real)0;
    ppid[k] = valid ? __ldg(src.pid + i) : 0u;
  }
  if (threadIdx.x == 0) {
    s_lo = 0xFFFFFFFFu;
    s_hi = 0;
  }
  for (int i = threadIdx.x; i < TB_SPAN; i += TB_THREADS) s_cnt[i] = 0;
  __syncthreads();
  block_key_range(t, &s_lo, &s_hi);
  __syncthreads();
  const uint32_t lo = s_lo;
  const bool local = s_hi - lo < (uint32_t)TB_SPAN;
  uint32_t pos[TB_PER_THREAD];
  if (local) {
    // rank within the block's tile: one shared atomic per group of equal keys
#pragma unroll
    for (int k = 0; k < TB_PER_THREAD; ++k) {
      const unsigned peers = __match_any_sync(0xffffffffu, t[k]);
      const int leader = __ffs(peers) - 1;
      uint32_t b = 0;
      if (t[k] != 0xFFFFFFFFu && lane == leader) b = atomicAdd(&s_cnt[t[k] - lo], (uint32_t)__popc(peers));
      pos[k] = __shfl_sync(0xffffffffu, b, leader) + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    // per tile: the block's global base (one atomic per non-empty tile) and
    // the local start (exclusive scan of the counts, four tiles per thread)
    static_assert(TB_SPAN == 4 * TB_THREADS, "four tiles per thread");
    uint32_t cnt4[4], run = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = 4 * threadIdx.x + j;
      cnt4[j] = s_cnt[i];
      if (cnt4[j]) s_base[i] = atomicAdd(&cursor[lo + i], cnt4[j]);
      run += cnt4[j];
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_wsum[w];
    uint32_t start = wbase + incl - run;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s_cnt[4 * threadIdx.x + j] = start;
      start += cnt4[j];
    }
    __syncthreads();
    if constexpr (ScatterStage<real, D>::on) {
      real* su = reinterpret_cast<real*>(smem_raw);  // [2D+1][TB_ITEMS]: u, v, w
      uint32_t* spid = reinterpret_cast<uint32_t*>(su + (size_t)(2 * D + 1) * TB_ITEMS);
      uint32_t* sdst = spid + TB_ITEMS;
#pragma unroll
      for (int k = 0; k < TB_PER_THREAD; ++k) {
        const size_t i = chunk + (size_t)k * TB_THREADS + threadIdx.x;
        if (i < np) {
          const uint32_t ti = t[k] - lo;
          const uint32_t L = s_cnt[ti] + pos[k];
#pragma unroll
          for (int m = 0; m < D; ++m) {
            su[(size_t)m * TB_ITEMS + L] = pu[k][m];
            su[(size_t)(D + m) * TB_ITEMS + L] = pv[k][m];
          }
          su[(size_t)(2 * D) * TB_ITEMS + L] = pw[k];
          spid[L] = ppid[k];
          sdst[L] = s_base[ti] + pos[k];
        }
      }
      __syncthreads();
      const int nvalid = (int)min((size_t)TB_ITEMS, np - chunk);
      for (int j = threadIdx.x; j < nvalid; j += TB_THREADS) {
        const uint32_t p = sdst[j];
#pragma unroll
        for (int m = 0; m < D; ++m) {
          dst.u[m][p] = su[(size_t)m * TB_ITEMS + j];
          dst.v[m][p] = su[(size_t)(D + m) * TB_ITEMS + j];
        }
        dst.w[p] = su[(size_t)(2 * D) * TB_ITEMS + j];
        dst.pid[p] = spid[j];
      }
      return;
    } else {
#pragma unroll
      for (int k = 0; k < TB_PER_THREAD; ++k)
        if (t[k] != 0xFFFFFFFFu) pos[k] += s_base[t[k] - lo];
    }
  } else {
#pragma unroll
    for (int k = 0; k < TB_PER_THREAD; ++k) {
      const bool valid = t[k] != 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xffffffffu, t[k]);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (valid && lane == leader) base = atomicAdd(&cursor[t[k]], (uint32_t)__popc(peers));
      pos[k] = __shfl_sync(0xffffffffu, base, leader) + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
  }
  // direct move of the payload loaded at the start
#pragma unroll
  for (int k = 0; k < TB_PER_THREAD; ++k) {
    const size_t i = chunk + (size_t)k * TB_THREADS + threadIdx.x;
    if (i >= np) continue;
    const uint32_t p = pos[k];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      dst.u[m][p] = pu[k][m];
      dst.v[m][p] = pv[k][m];
    }
    dst.w[p] = pw[k];
    dst.pid[p] = ppid[k];
  }
}

template <typename real, int D>
int launch_tile_scatter(const PArrays<real, D>& src, const PArrays<real, D>& dst, const uint32_t* keys,
                        uint32_t* cursor, size_t np, cudaStream_t s) {
  if (np == 0) return SG_OK;
  const size_t smem = ScatterStage<real, D>::on ? ScatterStage<real, D>::bytes : 0;
  static bool attr_set = false;
  if (!attr_set && smem > 0) {  // with the static counters the total may pass 48 KB
    SG_CUDA(cudaFuncSetAttribute(k_tile_scatter<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  k_tile_scatter<real, D><<<(unsigned)((np + TB_ITEMS - 1) / TB_ITEMS), TB_THREADS, smem, s>>>(src, dst, keys,
                                                                                              cursor, np);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

__global__ void __launch_bounds__(256) k_counts(const uint32_t* keys, size_t np, uint32_t* counts) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = i < np;
  uint32_t k = valid ? keys[i] : 0xFFFFFFFFu;
  unsigned peers = __match_any_sync(0xffffffffu, k);
  if (valid && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[k], (uint32_t)__popc(peers));
}

int launch_counts(const uint32_t* keys, size_t np, uint32_t* counts, cudaStream_t s) {
  if (np == 0) return SG_OK;
  k_counts<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(keys, np, counts);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_SORT(real, D)                                                                           \
  template int launch_keys<real, D>(const PArrays<real, D>&, size_t, int, uint32_t*, uint32_t*,        \
                                    unsigned long long*, unsigned*, cudaStream_t);                      \
  template int launch_keys_raw<real, D>(const real* const*, size_t, int, uint32_t*, uint32_t*,         \
                                        unsigned long long*, unsigned*, cudaStream_t);                  \
  template int launch_permute<real, D>(const PArrays<real, D>&, const PArrays<real, D>&, const uint32_t*, \
                                       size_t, cudaStream_t);                                             \
  template int launch_unpermute<real, D>(const PArrays<real, D>&, const PArrays<real, D>&, size_t, cudaStream_t); \
  template int launch_tile_keys<real, D>(const PArrays<real, D>&, size_t, int, const SortFuse&, unsigned*,         \
                                         cudaStream_t);                                                            \
  template int launch_tile_scatter<real, D>(const PArrays<real, D>&, const PArrays<real, D>&, const uint32_t*,     \
                                            uint32_t*, size_t, cudaStream_t);

SG_INST_SORT(float, 2)
SG_INST_SORT(float, 3)
SG_INST_SORT(double, 2)
SG_INST_SORT(double, 3)

}  // namespace sg
