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
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 16;
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

// Per-tile counts of the keys: each warp reads TS_ROUNDS x 32 keys (vectors
// of four), combines equal keys within the warp and adds the group counts.
constexpr int TS_ROUNDS = 8;

__global__ void __launch_bounds__(256) k_tile_hist(const uint32_t* __restrict__ keys, size_t np,
                                                   uint32_t* tile_count) {
  const int lane = threadIdx.x & 31;
  const size_t wbase = ((size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (128 * (TS_ROUNDS / 4));
#pragma unroll
  for (int r = 0; r < TS_ROUNDS / 4; ++r) {
    const size_t i0 = wbase + ((size_t)r * 32 + lane) * 4;
    uint32_t t[4];
    if (i0 + 4 <= np) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(keys + i0));
      t[0] = v.x;
      t[1] = v.y;
      t[2] = v.z;
      t[3] = v.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) t[k] = i0 + k < np ? keys[i0 + k] : 0xFFFFFFFFu;
    }
    uint32_t c0 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (t[k] == t[0])
        ++c0;
      else if (t[k] != 0xFFFFFFFFu)
        atomicAdd(&tile_count[t[k]], 1u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, t[0]);
    const uint32_t sum = __reduce_add_sync(peers, c0);
    if (t[0] != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&tile_count[t[0]], sum);
  }
}

int launch_tile_hist(const uint32_t* keys, size_t np, uint32_t* tile_count, cudaStream_t s) {
  if (np == 0) return SG_OK;
  const size_t per_block = (size_t)256 * TS_ROUNDS;  // 8 warps x (TS_ROUNDS / 4) rounds x 128 keys
  k_tile_hist<<<(unsigned)((np + per_block - 1) / per_block), 256, 0, s>>>(keys, np, tile_count);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// Scatter every particle to its tile's next free slot.  Each warp takes
// TS_ROUNDS x 32 consecutive particles: it reserves the slots of all rounds
// (lanes with equal tiles share one reservation) and loads all payloads
// before storing any, so the round trips overlap.  Within a tile the order
// follows the warps' arrival: the step sort is a valid, not a stable,
// counting sort by tile key.
template <typename real, int D>
__global__ void __launch_bounds__(256) k_tile_scatter(PArrays<real, D> src, PArrays<real, D> dst,
                                                      const uint32_t* __restrict__ keys, uint32_t* cursor,
                                                      size_t np) {
  constexpr int R = 4;
  const int lane = threadIdx.x & 31;
  const size_t wbase = ((size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 * R);
  uint32_t base[R], rank[R];
  int leader[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const size_t i = wbase + (size_t)r * 32 + lane;
    const bool valid = i < np;
    const uint32_t t = valid ? __ldg(keys + i) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    leader[r] = __ffs(peers) - 1;
    rank[r] = (uint32_t)__popc(peers & ((1u << lane) - 1u));
    base[r] = 0;
    if (valid && lane == leader[r]) base[r] = atomicAdd(&cursor[t], (uint32_t)__popc(peers));
  }
  real pu[R][D], pv[R][D], pw[R];
  uint32_t pid[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const size_t i = wbase + (size_t)r * 32 + lane;
    const bool valid = i < np;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      pu[r][m] = valid ? __ldg(src.u[m] + i) : (real)0;
      pv[r][m] = valid ? __ldg(src.v[m] + i) : (real)0;
    }
    pw[r] = valid ? __ldg(src.w + i) : (real)0;
    pid[r] = valid ? __ldg(src.pid + i) : 0u;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t pos = __shfl_sync(0xffffffffu, base[r], leader[r]) + rank[r];
    const size_t i = wbase + (size_t)r * 32 + lane;
    if (i >= np) continue;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      dst.u[m][pos] = pu[r][m];
      dst.v[m][pos] = pv[r][m];
    }
    dst.w[pos] = pw[r];
    dst.pid[pos] = pid[r];
  }
}

template <typename real, int D>
int launch_tile_scatter(const PArrays<real, D>& src, const PArrays<real, D>& dst, const uint32_t* keys,
                        uint32_t* cursor, size_t np, cudaStream_t s) {
  if (np == 0) return SG_OK;
  const size_t per_block = (size_t)256 * 4;
  k_tile_scatter<real, D><<<(unsigned)((np + per_block - 1) / per_block), 256, 0, s>>>(src, dst, keys, cursor, np);
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
