// CIC charge deposition onto the regular level-n grid through a
// shared-memory window per particle chunk, and the restriction that carries
// the regular density to every component grid.
//
// Proposition 1 (Section 4.1, Appendix A): for node-centred grids and linear
// shapes, depositing on the regular grid and then applying R_i
// (eq. restriction) gives exactly the direct deposit onto component grid i.
// The GPU therefore deposits 2^d corners per particle once and restricts,
// instead of 2^d * n_c scattered adds per particle.
#include <limits.h>

#include <algorithm>

#include "sg_kernels.cuh"

namespace sg {

// Shared-memory accumulator of the deposit window.
//
// FP32 path: 32-bit fixed point, so the window uses native integer shared
// atomics and its sums do not depend on the order of the adds.  The scale is
// the power of two 2^(20 - E) with max_p |q_p| / V <= 2^E (1 - 2^-11) over
// the run's particles (set at upload): one contribution rounds to at most
// 2^20 - 2^9 in magnitude, and DEP_CHUNK = 2^11 of them stay below
// 2^31 - 2^20, so no node overflows.  A contribution is rounded once, to
// 2^-20 of the largest charge.  Because |x| < 2^22, x + 1.5 * 2^23 lands in
// [2^23, 2^24), where the float spacing is 1: its low mantissa bits are
// round-to-nearest-even(x), with no conversion instruction.
//
// FP64 path: plain double and no scaling.
static_assert(DEP_CHUNK <= 2048, "the fixed-point scale assumes at most 2^11 particles per window");
template <typename real>
struct WinAcc;
template <>
struct WinAcc<float> {
  using T = int;
  static constexpr bool fixed = true;
  static __device__ __forceinline__ T quantize_fma(float a, float b) {
    return __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4B400000;
  }
  static __device__ __forceinline__ float value(T s, float inv_scale) { return (float)s * inv_scale; }
};
template <>
struct WinAcc<double> {
  using T = double;
  static constexpr bool fixed = false;
  static __device__ __forceinline__ T quantize_fma(double a, double b) { return a * b; }
  static __device__ __forceinline__ double value(T s, double) { return s; }
};

// Index of the node left of a scaled coordinate s = u * 2^n - shift in
// [-1/2, 2^n) (shift = 1/2 on cell-centred grids, where node k sits at
// u = (k + 1/2) / 2^n), wrapped periodically, and the offset from it.
// FP32: floor through the same 1.5 * 2^23 rounding (ties at exact integers
// may land on the node below with offset 1, which deposits identical
// weights on identical nodes); FP64: floor.
__device__ __forceinline__ void cell_frac(float s, int mask, int& c, float& f) {
  const float t = (s - 0.5f) + 12582912.0f;
  const float fl = t - 12582912.0f;
  c = (__float_as_int(t) - 0x4B400000) & mask;
  f = s - fl;
}
__device__ __forceinline__ void cell_frac(double s, int mask, int& c, double& f) {
  const double fl = floor(s);
  c = (int)fl & mask;
  f = s - fl;
}

// ---------------------------------------------------------------- deposit
//
// Persistent blocks walk chunks of DEP_CHUNK consecutive particles
// (consecutive in tile-key order after a sort, so a chunk covers a compact
// group of cells).  Per chunk every thread reads the chunk's middle particle
// and takes its cell as the anchor of a fixed window of side^d regular nodes
// centred on it; its four particles (16-byte vector loads) add their CIC
// weights into the window when all 2^d corners fall inside, else straight to
// the global grid.  The window's touched box is then added to the global
// grid row by row and cleared for the next chunk: two block barriers per
// chunk, no reductions before the adds.  FP32: the window's x origin is a
// multiple of 4 and its side a multiple of 4, so each lane moves four
// nodes with one 16-byte shared load and one vector global add
// (red.global.add.v4.f32), skipping groups that are all zero; this matters
// most a few steps after a sort, when the particles of a chunk have spread
// and the touched box has grown.  FP64: one atomic add per non-zero node.
//
// FP32: WinAcc fixed point with the run's scale 2^(20 - E), max_p |q_p|/V <=
// 2^E (1 - 2^-11) (set at upload; charges do not change), so a window of at
// most 2^11 particles cannot overflow.  FP64: plain double, scale 1.
template <typename real, int D>
__global__ void __launch_bounds__(DEP_THREADS) k_deposit(PArrays<real, D> p, size_t np, int n,
                                                         real inv_cell_vol, real* __restrict__ rho, int side,
                                                         real scale, real inv_scale, real shift) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using W = WinAcc<real>;
  using T = typename W::T;
  T* win = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_box[2][2 * D];  // per chunk parity: lo[D], hi[D] of the touched window
  const int N = 1 << n;
  const int mask = N - 1;
  const int lane = threadIdx.x & 31;
  const int half = side >> 1;
  int nwin = 1;
#pragma unroll
  for (int m = 0; m < D; ++m) nwin *= side;
  pdl_trigger();  // the restriction may start launching
  {
    uint4* w4 = reinterpret_cast<uint4*>(smem_raw);
    const int n4 = (int)((nwin * sizeof(T) + 15) / 16);
    for (int i = threadIdx.x; i < n4; i += DEP_THREADS) w4[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x < 2 * D) {
      s_box[0][threadIdx.x] = threadIdx.x < D ? INT_MAX : INT_MIN;
      s_box[1][threadIdx.x] = threadIdx.x < D ? INT_MAX : INT_MIN;
    }
  }
  const size_t nchunks = (np + DEP_CHUNK - 1) / DEP_CHUNK;
  int par = 0;
  for (size_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, par ^= 1) {
    const size_t chunk = ch * DEP_CHUNK;
    // ---- this thread's particles: DEP_ITEMS / 4 vectors of four
    real ub[DEP_ITEMS][D], qb[DEP_ITEMS];
#pragma unroll
    for (int j = 0; j < DEP_ITEMS / 4; ++j) {
      const size_t i0 = chunk + ((size_t)j * DEP_THREADS + threadIdx.x) * 4;
      if (i0 + 4 <= np) {
#pragma unroll
        for (int m = 0; m < D; ++m) {
          const V4<real> t = ld4(p.u[m] + i0);
#pragma unroll
          for (int k = 0; k < 4; ++k) ub[4 * j + k][m] = t.x[k];
        }
        const V4<real> t = ld4(p.w + i0);
#pragma unroll
        for (int k = 0; k < 4; ++k) qb[4 * j + k] = t.x[k] * inv_cell_vol;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool ok = i0 + k < np;
#pragma unroll
          for (int m = 0; m < D; ++m) ub[4 * j + k][m] = ok ? p.u[m][i0 + k] : (real)0;
          qb[4 * j + k] = ok ? p.w[i0 + k] * inv_cell_vol : (real)0;
        }
      }
    }
    // ---- anchor: the cell of the chunk's middle (or last) particle, read by every thread
    int anchor[D];
    {
      size_t mid = chunk + DEP_CHUNK / 2;
      if (mid >= np) mid = np - 1;
#pragma unroll
      for (int m = 0; m < D; ++m) anchor[m] = cell_of(__ldg(p.u[m] + mid), n, N);
    }
    // window origin (global node of window index 0) per axis; along x a
    // multiple of 4, so that 4 consecutive window nodes are 4 aligned global
    // nodes (16-byte vector adds in the flush)
    int origin[D];
#pragma unroll
    for (int m = 0; m < D; ++m) origin[m] = (anchor[m] - half) & mask;
    origin[0] &= ~3;
    __syncthreads();  // the previous chunk's flush has cleared the window
    if (threadIdx.x < 2 * D) s_box[par ^ 1][threadIdx.x] = threadIdx.x < D ? INT_MAX : INT_MIN;
    int lo[D], hi[D];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      lo[m] = INT_MAX;
      hi[m] = INT_MIN;
    }
#pragma unroll
    for (int it = 0; it < DEP_ITEMS; ++it) {
      if (qb[it] == (real)0) continue;
      int c[D], l[D];
      real f[D];
      bool fast = true;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        cell_frac(ub[it][m] * (real)N - shift, mask, c[m], f[m]);
        l[m] = (c[m] - origin[m]) & mask;
        fast &= l[m] + 1 < side;
      }
      if (fast) {
        const real qs = qb[it] * scale;
        const real wx0 = (real)1 - f[0], wx1 = f[0];
        if (D == 2) {
          const int base = l[0] + side * l[1 % D];
          const real a = qs * ((real)1 - f[1 % D]), b = qs * f[1 % D];
          atomicAdd(&win[base], W::quantize_fma(a, wx0));
          atomicAdd(&win[base + 1], W::quantize_fma(a, wx1));
          atomicAdd(&win[base + side], W::quantize_fma(b, wx0));
          atomicAdd(&win[base + side + 1], W::quantize_fma(b, wx1));
        } else {
          const int sz = side * side;
          const int base = l[0] + side * l[1 % D] + sz * l[D - 1];
          const real wy[2] = {(real)1 - f[1 % D], f[1 % D]};
          const real wz[2] = {(real)1 - f[D - 1], f[D - 1]};
#pragma unroll
          for (int kz = 0; kz < 2; ++kz)
#pragma unroll
            for (int ky = 0; ky < 2; ++ky) {
              const real a = qs * wz[kz] * wy[ky];
              const int o = base + kz * sz + ky * side;
              atomicAdd(&win[o], W::quantize_fma(a, wx0));
              atomicAdd(&win[o + 1], W::quantize_fma(a, wx1));
            }
        }
#pragma unroll
        for (int m = 0; m < D; ++m) {
          lo[m] = min(lo[m], l[m]);
          hi[m] = max(hi[m], l[m] + 1);
        }
      } else {  // a corner outside the window: all corners to the global grid
#pragma unroll 1
        for (int corner = 0; corner < (1 << D); ++corner) {
          real wgt = qb[it];
          size_t g = 0, gs = 1;
#pragma unroll
          for (int m = 0; m < D; ++m) {
            const int bb = (corner >> m) & 1;
            wgt *= bb ? f[m] : ((real)1 - f[m]);
            g += (size_t)((c[m] + bb) & mask) * gs;
            gs *= (size_t)N;
          }
          atomicAdd(&rho[g], wgt);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < D; ++m) {
      lo[m] = __reduce_min_sync(0xffffffffu, lo[m]);
      hi[m] = __reduce_max_sync(0xffffffffu, hi[m]);
    }
    if (lane == 0) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        atomicMin(&s_box[par][m], lo[m]);
        atomicMax(&s_box[par][D + m], hi[m]);
      }
    }
    __syncthreads();  // the chunk's window is complete
    int blo[D], bhi[D];
    bool any = true;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      blo[m] = s_box[par][m];
      bhi[m] = s_box[par][D + m];
      any &= blo[m] <= bhi[m];
    }
    if (any) {  // the touched box: add to the grid and clear
      // The box's (row, x) items are spread over all the block's threads,
      // consecutive threads along x, so that narrow boxes (3D, or right
      // after a sort) keep every lane busy.  FP32: an item is four nodes
      // (one 16-byte shared load, one vector add); FP64: one node.
      const int ny = bhi[1 % D] - blo[1 % D] + 1;
      const int nrows = D == 2 ? ny : ny * (bhi[D - 1] - blo[D - 1] + 1);
      constexpr int PER = W::fixed ? 4 : 1;
      const int x0 = W::fixed ? (blo[0] & ~3) : blo[0];
      const int nx = (bhi[0] - x0) / PER + 1;
      const int total = nrows * nx;
      for (int f = threadIdx.x; f < total; f += DEP_THREADS) {
        const int r = f / nx;
        const int x = x0 + (f - r * nx) * PER;
        const int ly = blo[1 % D] + (D == 2 ? r : r % ny);
        const int lz = D == 2 ? 0 : blo[D - 1] + r / ny;
        const size_t gy = (size_t)((origin[1 % D] + ly) & mask);
        const size_t grow = D == 2 ? gy * N : ((size_t)((origin[D - 1] + lz) & mask) * N + gy) * N;
        T* wrow = win + ((size_t)lz * side + ly) * side;
        if constexpr (W::fixed) {
          const int4 v = *reinterpret_cast<const int4*>(wrow + x);
          if ((v.x | v.y | v.z | v.w) != 0) {
            float* dst = rho + grow + ((origin[0] + x) & mask);
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst),
                         "f"(W::value(v.x, inv_scale)), "f"(W::value(v.y, inv_scale)),
                         "f"(W::value(v.z, inv_scale)), "f"(W::value(v.w, inv_scale))
                         : "memory");
            *reinterpret_cast<int4*>(wrow + x) = make_int4(0, 0, 0, 0);
          }
        } else {
          const T v = wrow[x];
          if (v != (T)0) {
            atomicAdd(&rho[grow + ((origin[0] + x) & mask)], W::value(v, inv_scale));
            wrow[x] = (T)0;
          }
        }
      }
    }
  }
}

template <typename real, int D>
int launch_deposit(const PArrays<real, D>& p, size_t np, int n, real inv_cell_vol, real* rho, int win_cap_nodes,
                   real scale, real inv_scale, real shift, cudaStream_t s) {
  if (np == 0) return SG_OK;
  if (n < 2) {  // the flush adds groups of 4 aligned nodes of a row
    set_error("deposit: level n must be at least 2");
    return SG_ERR_UNSUPPORTED;
  }
  using T = typename WinAcc<real>::T;
  const long long cap = (long long)win_cap_nodes * 8 / (long long)sizeof(T);  // same bytes for either type
  int side = 4;  // largest multiple of 4 with side^D <= capacity (16-byte window rows)
  while (true) {
    long long nxt = 1;
    for (int m = 0; m < D; ++m) nxt *= (side + 4);
    if (nxt > cap) break;
    side += 4;
  }
  long long nodes = 1;
  for (int m = 0; m < D; ++m) nodes *= side;
  const size_t smem = ((size_t)nodes * sizeof(T) + 15) / 16 * 16;  // zeroed in 16-byte words
  if (smem > 200 * 1024) {
    set_error("deposit: window capacity above 200 KB of shared memory");
    return SG_ERR_UNSUPPORTED;
  }
  // resident blocks per SM for each window size met so far (the autotuner
  // tries several capacities; the answer depends on the window's bytes)
  static bool attr_set = false;
  static size_t known_smem[8];
  static int known_per_sm[8];
  static int nknown = 0;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_deposit<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    SG_CUDA(cudaFuncSetAttribute(k_deposit<real, D>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr_set = true;
  }
  int per_sm = 0;
  for (int i = 0; i < nknown; ++i)
    if (known_smem[i] == smem) per_sm = known_per_sm[i];
  if (!per_sm) {
    SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deposit<real, D>, DEP_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    if (nknown < 8) {
      known_smem[nknown] = smem;
      known_per_sm[nknown] = per_sm;
      ++nknown;
    }
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const size_t nchunks = (np + DEP_CHUNK - 1) / DEP_CHUNK;
  const unsigned blocks = (unsigned)std::min<size_t>(nchunks, (size_t)sms * per_sm);
  k_deposit<real, D><<<blocks, DEP_THREADS, smem, s>>>(p, np, n, inv_cell_vol, rho, side, scale, inv_scale, shift);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// ---------------------------------------------------------------- restriction
//
// R_i of eq. restriction is separable: along one axis, restricting a line
// from level l to l-1 is full weighting b[k] = (a[2k-1] + 2 a[2k] + a[2k+1]) / 4
// (periodic), which is (h_l / h_{l-1}) sum_k' W_{l-1}(x_k - x_k') a[k'].
// Composing the steps is exact because a coarse hat is linear between the
// finer nodes (Appendix A).
//
// Cell-centred grids (node k at (k + 1/2) h): the coarse hat is no longer
// linear between fine nodes and the steps do not compose; R from level n
// to level l (r = 2^(n-l) fine cells per coarse cell) weights fine value j
// by (1/r) max(0, 1 - |j + 1/2 - (k + 1/2) r| / r).  It still factors
// into the same cascade: average neighbouring values onto the cell faces,
// a[t] = (x[t-1] + x[t]) / 2 (the faces are the nodes of a node-centred
// level-n line), apply full weighting n-l-1 times, and take the last step's
// full weighting at the odd nodes instead of the even ones,
// R_l x[k] = (a[2k] + 2 a[2k+1] + a[2k+2]) / 4.  (The cell-centred
// prolongation is linear interpolation through the coarse centres; R is
// (h / h_l) times its transpose, and the prolongation is the node-centred
// one from level l+1, whose odd nodes are the coarse centres and even nodes
// their midpoints, sampled at the fine centres, which are the midpoints of
// the level-n nodes.)  So one register cascade serves every level again:
// at each step the even full weighting carries the cascade and the odd one
// is the output.
//
// Arrays keep their natural layout [outer][len][inner] (inner = the axes
// already restricted, contiguous; len = the axis being restricted).  One
// warp restricts one line of 2^top values held in registers (VPL
// consecutive values per lane): each halving step needs one shuffle for the
// left neighbour's last value while a lane holds more than one value, then
// three shuffles per step once the line fits in one value per lane.  Lines
// along the contiguous axis (inner = 1) are read straight from global
// memory; the others go through a shared-memory tile of up to 8 adjacent
// lines, filled with 32-byte row segments.  Every requested level is
// written to dst[(o * 2^l + j) * inner + i] for value j of line (o, i).

// Shared-memory index of value t of a tile row: 4 padding words after every
// 32, so lanes that read runs of consecutive values hit distinct banks.
__device__ __forceinline__ int rj_pad(int t) { return t + ((t >> 5) << 2); }

template <typename real>
struct RjOut {
  const LineJob* J;
  size_t o;  // outer index of this warp's line
  int i;     // inner index
  int lane;
  template <int V>
  __device__ __forceinline__ void emit(const real* v, int level) const {
    if (!((J->tmask >> level) & 1)) return;
    real* d = reinterpret_cast<real*>(J->dst[level]);
    const size_t inner = (size_t)J->inner;
    const size_t row0 = o << level;
    if (inner == 1 && V >= 4 && sizeof(real) == 4) {
      float* df = reinterpret_cast<float*>(d) + row0 + (size_t)lane * V;
#pragma unroll
      for (int k = 0; k < V; k += 4)
        *reinterpret_cast<float4*>(df + k) = make_float4((float)v[k], (float)v[k + 1], (float)v[k + 2], (float)v[k + 3]);
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) d[(row0 + (size_t)lane * V + k) * inner + i] = v[k];
    }
  }
};

template <typename real, int V>
struct RjLevels {
  // v[0..V) are this lane's V consecutive values of the current level.
  static __device__ __forceinline__ void run(real* v, int& level, int tmin, const RjOut<real>& e) {
    const real left = __shfl_sync(0xffffffffu, v[V - 1], (e.lane + 31) & 31);
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {  // in place: v[k] is written after its last read
      const real am = (k == 0) ? left : v[2 * k - 1];
      v[k] = (real)0.25 * am + (real)0.5 * v[2 * k] + (real)0.25 * v[2 * k + 1];
    }
    --level;
    e.template emit<V / 2>(v, level);
    if (level > tmin) RjLevels<real, V / 2>::run(v, level, tmin, e);
  }
};
template <typename real>
struct RjLevels<real, 1> {
  static __device__ __forceinline__ void run(real*, int&, int, const RjOut<real>&) {}
};

// Cell-centred cascade: v[0..V) are this lane's V consecutive face values of
// the current level; emits the odd full weighting (the cell-centred
// restriction to the next level down) and keeps the even one.
template <typename real, int V>
struct RjLevelsCell {
  static __device__ __forceinline__ void run(real* v, int& level, int tmin, const RjOut<real>& e) {
    const real left = __shfl_sync(0xffffffffu, v[V - 1], (e.lane + 31) & 31);
    const real right = __shfl_sync(0xffffffffu, v[0], (e.lane + 1) & 31);
    real ob[V / 2];
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {  // in place: v[k] is written after its last read
      const real am = (k == 0) ? left : v[2 * k - 1];
      const real a0 = v[2 * k], a1 = v[2 * k + 1];
      const real a2 = (k == V / 2 - 1) ? right : v[2 * k + 2];
      ob[k] = (real)0.25 * a0 + (real)0.5 * a1 + (real)0.25 * a2;
      v[k] = (real)0.25 * am + (real)0.5 * a0 + (real)0.25 * a1;
    }
    --level;
    e.template emit<V / 2>(ob, level);
    if (level > tmin) RjLevelsCell<real, V / 2>::run(v, level, tmin, e);
  }
};
template <typename real>
struct RjLevelsCell<real, 1> {
  static __device__ __forceinline__ void run(real*, int&, int, const RjOut<real>&) {}
};

template <typename real, int VPL>
__device__ __forceinline__ void rj_load_run(const real* p, real* v) {
  if (VPL >= 4 && sizeof(real) == 4) {
#pragma unroll
    for (int k = 0; k < VPL; k += 4) {
      const float4 t = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(p) + rj_pad(k));
      v[k] = (real)t.x;
      v[k + 1] = (real)t.y;
      v[k + 2] = (real)t.z;
      v[k + 3] = (real)t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < VPL; ++k) v[k] = p[rj_pad(k)];
  }
}

template <typename real, int VPL, bool CELL>
__global__ void __launch_bounds__(256) k_restrict_warp(const LineJob* __restrict__ jobs, int njobs, real mean) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* tile = reinterpret_cast<real*>(smem_raw);
  pdl_trigger();
  const int jb = find_job(jobs, njobs);  // job tables are written once, at set-up
  const LineJob* J = jobs + jb;
  pdl_wait();
  const int lpb = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int top = J->top, len = 1 << top;
  const int inner = J->inner;
  const int b = blockIdx.x - J->block_begin;
  const real* src = reinterpret_cast<const real*>(J->src);
  real v[VPL];
  size_t o;
  int i;
  bool active;
  if (inner == 1) {  // contiguous lines: one per warp, straight from global memory
    o = (size_t)b * lpb + w;
    i = 0;
    active = o < (size_t)J->outer;
    if (active) {
      const real* line = src + o * (size_t)len;
      if (VPL >= 4) {
#pragma unroll
        for (int k = 0; k < VPL; k += 4) {
          const V4<real> t = ld4(line + lane * VPL + k);
#pragma unroll
          for (int q = 0; q < 4; ++q) v[k + q] = t.x[q];
        }
      } else if (VPL == 2) {
        v[0] = line[2 * lane];
        v[VPL - 1] = line[2 * lane + 1];
      } else {
        v[0] = lane < len ? line[lane] : (real)0;
      }
    }
  } else {  // strided lines: a tile of cpb adjacent lines through shared memory
    const int cpb = min(lpb, inner);  // both powers of two
    const int per_o = inner / cpb;
    o = (size_t)(b / per_o);
    const int i0 = (b % per_o) * cpb;
    i = i0 + w;
    active = w < cpb;
    const int S = J->tile_stride;
    const int logc = __ffs(cpb) - 1;
    const real* base = src + o * (size_t)len * inner + i0;
    if (sizeof(real) == 4 && cpb >= 4) {
      // 16-byte row pieces, eight loads in flight per thread
      const int q = cpb >> 2, logq = __ffs(q) - 1;
      const int total = len << logq;
      for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {
        float4 tv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < total) {
            const int c4 = (e & (q - 1)) << 2, t = e >> logq;
            tv[u] = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(base) + (size_t)t * inner + c4));
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < total) {
            const int c4 = (e & (q - 1)) << 2, t = e >> logq;
            const int p = rj_pad(t);
            tile[(c4 + 0) * S + p] = (real)tv[u].x;
            tile[(c4 + 1) * S + p] = (real)tv[u].y;
            tile[(c4 + 2) * S + p] = (real)tv[u].z;
            tile[(c4 + 3) * S + p] = (real)tv[u].w;
          }
        }
      }
    } else {
      const int total = len << logc;
      for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {
        real tv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < total) tv[u] = base[(size_t)(e >> logc) * inner + (e & (cpb - 1))];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < total) tile[(e & (cpb - 1)) * S + rj_pad(e >> logc)] = tv[u];
        }
      }
    }
    __syncthreads();
    if (active) {
      if (VPL > 1 || top >= 5) {
        rj_load_run<real, VPL>(tile + w * S + rj_pad(lane * VPL), v);
      } else {
        v[0] = lane < len ? tile[w * S + lane] : (real)0;
      }
    }
  }
  if (!active) return;  // no block-wide barrier follows
  if (J->sub_mean) {
#pragma unroll
    for (int k = 0; k < VPL; ++k) v[k] -= mean;
  }
  const RjOut<real> e{J, o, i, lane};
  int level = top;
  const int tmin = J->tmin;
  if (VPL > 1 || top >= 5) {
    e.template emit<VPL>(v, level);
    if (CELL) {  // onto the faces: a[t] = (x[t-1] + x[t]) / 2, periodic over the whole line
      const real left = __shfl_sync(0xffffffffu, v[VPL - 1], (lane + 31) & 31);
#pragma unroll
      for (int k = VPL - 1; k > 0; --k) v[k] = (real)0.5 * (v[k - 1] + v[k]);
      v[0] = (real)0.5 * (left + v[0]);
      if (level > tmin) RjLevelsCell<real, VPL>::run(v, level, tmin, e);
    } else {
      if (level > tmin) RjLevels<real, VPL>::run(v, level, tmin, e);
    }
  } else {  // a line shorter than a warp
    if (((J->tmask >> level) & 1) && lane < len)
      reinterpret_cast<real*>(J->dst[level])[((o << level) + lane) * (size_t)inner + i] = v[0];
    if (CELL) {
      const real left = __shfl_sync(0xffffffffu, v[0], (lane - 1) & (len - 1));
      v[0] = (real)0.5 * (left + v[0]);
    }
  }
  // one value per lane on m = 2^level lanes
  real a = v[0];
  while (level > tmin) {
    const int m = 1 << level, h = m >> 1;
    const int k = lane & (h - 1);
    const real am = __shfl_sync(0xffffffffu, a, (2 * k - 1) & (m - 1));
    const real a0 = __shfl_sync(0xffffffffu, a, (2 * k) & (m - 1));
    const real ap = __shfl_sync(0xffffffffu, a, (2 * k + 1) & (m - 1));
    real out;
    if (CELL) {
      const real a2 = __shfl_sync(0xffffffffu, a, (2 * k + 2) & (m - 1));
      out = (real)0.25 * a0 + (real)0.5 * ap + (real)0.25 * a2;
    }
    a = (real)0.25 * am + (real)0.5 * a0 + (real)0.25 * ap;
    if (!CELL) out = a;
    --level;
    if (((J->tmask >> level) & 1) && lane < h)
      reinterpret_cast<real*>(J->dst[level])[((o << level) + lane) * (size_t)inner + i] = out;
  }
}

template <typename real>
int launch_restrict_pass(const LineJob* jobs_dev, int njobs, int nblocks, int lines_per_block, int vpl,
                         int smem_bytes, bool cell, real mean, cudaStream_t s) {
  if (njobs == 0 || nblocks == 0) return SG_OK;
  const unsigned threads = 32u * (unsigned)lines_per_block;
#define SG_RJ_LAUNCH(V, C)                                                                                   \
  {                                                                                                          \
    static bool attr_set = false;                                                                            \
    if (!attr_set) {                                                                                         \
      SG_CUDA(cudaFuncSetAttribute(k_restrict_warp<real, V, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   200 * 1024));                                                             \
      attr_set = true;                                                                                       \
    }                                                                                                        \
    SG_CUDA(launch_pdl(k_restrict_warp<real, V, C>, dim3(nblocks), dim3(threads), smem_bytes, s, jobs_dev,   \
                       njobs, mean));                                                                        \
  }
#define SG_RJ_CASE(V)            \
  case V:                        \
    if (cell)                    \
      SG_RJ_LAUNCH(V, true)      \
    else                         \
      SG_RJ_LAUNCH(V, false)     \
    break;
  switch (vpl) {
    SG_RJ_CASE(1)
    SG_RJ_CASE(2)
    SG_RJ_CASE(4)
    SG_RJ_CASE(8)
    SG_RJ_CASE(16)
    SG_RJ_CASE(32)
    SG_RJ_CASE(64)
    SG_RJ_CASE(128)
    default:
      set_error("restriction: unsupported line length");
      return SG_ERR_UNSUPPORTED;
  }
#undef SG_RJ_CASE
#undef SG_RJ_LAUNCH
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_DEP(real, D)                                                                  \
  template int launch_deposit<real, D>(const PArrays<real, D>&, size_t, int, real, real*, int, real, real, real, \
                                       cudaStream_t);

SG_INST_DEP(float, 2)
SG_INST_DEP(float, 3)
SG_INST_DEP(double, 2)
SG_INST_DEP(double, 3)
template int launch_restrict_pass<float>(const LineJob*, int, int, int, int, int, bool, float, cudaStream_t);
template int launch_restrict_pass<double>(const LineJob*, int, int, int, int, int, bool, double, cudaStream_t);

}  // namespace sg
