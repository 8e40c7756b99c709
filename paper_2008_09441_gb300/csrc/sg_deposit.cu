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

#include "sg_kernels.cuh"

namespace sg {

// Shared-memory accumulator of the deposit window.
//
// FP32 path: 32-bit fixed point, so the window uses native integer shared
// atomics and its sums do not depend on the order of the adds.  The scale is
// the power of two 2^(19 - E) with max_p |q_p| / V < 2^E over the chunk: one
// contribution is below 2^19 in magnitude, and DEP_CHUNK = 2^11 of them stay
// below 2^30, so no node overflows.  A contribution is rounded once, to
// 2^-19 of the chunk's largest charge (the same resolution a float has for
// a sum of 2^5 such charges).  Because |x| < 2^22, x + 1.5 * 2^23 lands in
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

// Cell index and offset of a scaled coordinate s = u * 2^n in [0, 2^n).
// FP32: floor through the same 1.5 * 2^23 rounding (ties at exact integers
// may land on the cell below with offset 1, which deposits identical
// weights on identical nodes); FP64: a plain truncation.
__device__ __forceinline__ void cell_frac(float s, int mask, int& c, float& f) {
  const float t = (s - 0.5f) + 12582912.0f;
  const float fl = t - 12582912.0f;
  c = (__float_as_int(t) - 0x4B400000) & mask;
  f = s - fl;
}
__device__ __forceinline__ void cell_frac(double s, int mask, int& c, double& f) {
  int ci = (int)s;
  ci = ci < 0 ? 0 : (ci > mask ? mask : ci);
  c = ci;
  f = s - (double)ci;
}

// ---------------------------------------------------------------- deposit
//
// Each block takes DEP_CHUNK consecutive particles (consecutive in tile-key
// order after a sort, so they occupy a compact block of cells).  All of them
// are loaded first (16-byte vector loads); the chunk's middle particle fixes
// the anchor cell and the periodic bounding box of the chunk's cells sizes a
// window of regular nodes in shared memory, accumulated with WinAcc.  The
// window is then added to the global grid row by row (coalesced atomics,
// zero nodes skipped).  Corners outside a window clamped to the
// shared-memory capacity add directly to the global grid.
template <typename real, int D>
__global__ void __launch_bounds__(DEP_THREADS) k_deposit(PArrays<real, D> p, size_t np, int n,
                                                         real inv_cell_vol, real* __restrict__ rho, int side) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using W = WinAcc<real>;
  using T = typename W::T;
  T* win = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_anchor[D], s_min[D], s_max[D];
  __shared__ unsigned s_qmax;
  const int N = 1 << n;
  const int mask = N - 1;
  const size_t chunk = (size_t)blockIdx.x * DEP_CHUNK;
  const int lane = threadIdx.x & 31;
  pdl_trigger();  // the restriction may start launching

  // ---- load the chunk: DEP_ITEMS / 4 vectors of four consecutive particles
  real ub[DEP_ITEMS][D], wb[DEP_ITEMS];
#pragma unroll
  for (int j = 0; j < DEP_ITEMS / 4; ++j) {
    const size_t i0 = chunk + ((size_t)j * DEP_THREADS + threadIdx.x) * 4;
    if (i0 + 4 <= np) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        V4<real> t = ld4(p.u[m] + i0);
#pragma unroll
        for (int k = 0; k < 4; ++k) ub[4 * j + k][m] = t.x[k];
      }
      V4<real> t = ld4(p.w + i0);
#pragma unroll
      for (int k = 0; k < 4; ++k) wb[4 * j + k] = t.x[k];
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ok = i0 + k < np;
#pragma unroll
        for (int m = 0; m < D; ++m) ub[4 * j + k][m] = ok ? p.u[m][i0 + k] : (real)0;
        wb[4 * j + k] = ok ? p.w[i0 + k] : (real)0;
      }
    }
  }
  // ---- anchor: the cell of the chunk's middle (or last) particle
  {
    size_t mid = chunk + DEP_CHUNK / 2;
    if (mid >= np) mid = np - 1;
    const int rel = (int)(mid - chunk);
    const int holder = (rel & (DEP_THREADS * 4 - 1)) >> 2;
    if ((int)threadIdx.x == holder) {
      const int item = 4 * (rel / (DEP_THREADS * 4)) + (rel & 3);
#pragma unroll
      for (int it = 0; it < DEP_ITEMS; ++it)
        if (it == item) {
#pragma unroll
          for (int m = 0; m < D; ++m) s_anchor[m] = cell_of(ub[it][m], n, N);
        }
    }
    if (threadIdx.x < D) {
      s_min[threadIdx.x] = INT_MAX;
      s_max[threadIdx.x] = INT_MIN;
    }
    if (threadIdx.x == 0) s_qmax = 0u;
  }
  __syncthreads();

  int c[DEP_ITEMS][D];
  real f[DEP_ITEMS][D];
  real q[DEP_ITEMS];
  int dmin[D], dmax[D];
  int anchor[D];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    dmin[m] = INT_MAX;
    dmax[m] = INT_MIN;
    anchor[m] = s_anchor[m];
  }
  unsigned qbits = 0u;  // max |q| as float bits (order-preserving for >= 0)
#pragma unroll
  for (int it = 0; it < DEP_ITEMS; ++it) {
    const size_t i = chunk + ((size_t)(it >> 2) * DEP_THREADS + threadIdx.x) * 4 + (it & 3);
    if (i < np) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        cell_frac(ub[it][m] * (real)N, mask, c[it][m], f[it][m]);
        const int dd = ((c[it][m] - anchor[m] + (N >> 1)) & mask) - (N >> 1);
        dmin[m] = min(dmin[m], dd);
        dmax[m] = max(dmax[m], dd);
      }
      q[it] = wb[it] * inv_cell_vol;
      if (W::fixed) qbits = max(qbits, __float_as_uint(fabsf((float)q[it])));
    } else {
      q[it] = (real)0;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        c[it][m] = anchor[m];
        f[it][m] = (real)0;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    dmin[m] = __reduce_min_sync(0xffffffffu, dmin[m]);
    dmax[m] = __reduce_max_sync(0xffffffffu, dmax[m]);
  }
  if (W::fixed) qbits = __reduce_max_sync(0xffffffffu, qbits);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < D; ++m) {
      atomicMin(&s_min[m], dmin[m]);
      atomicMax(&s_max[m], dmax[m]);
    }
    if (W::fixed) atomicMax(&s_qmax, qbits);
  }
  __syncthreads();

  // ---- window and fixed-point scale (every thread derives the same values)
  int org[D], ext[D];
  int nwin = 1;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    int lo = s_min[m];
    int e = s_max[m] - lo + 2;  // +1 node for the upper corner
    if (e >= N) {               // the window spans the whole axis
      e = N;
      lo = -(N >> 1);
    }
    if (e > side) {  // clamp around the anchor; outliers add to global
      e = side;
      lo = -(side >> 1);
    }
    org[m] = (anchor[m] + lo) & mask;
    ext[m] = e;
    nwin *= e;
  }
  real scale = (real)1, inv_scale = (real)1;
  if (W::fixed) {
    // max |q| < 2^E with E = (biased exponent) - 126; scale 2^(19 - E),
    // kept inside the normal float range.
    const int E = (int)(s_qmax >> 23) - 126;
    const int k = max(-126, min(127, 19 - E));
    scale = (real)__int_as_float((127 + k) << 23);
    inv_scale = (real)__int_as_float((127 - k) << 23);
  }
  {
    uint4* w4 = reinterpret_cast<uint4*>(smem_raw);
    const int n4 = (int)((nwin * sizeof(T) + 15) / 16);
    for (int i = threadIdx.x; i < n4; i += DEP_THREADS) w4[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();

#pragma unroll
  for (int it = 0; it < DEP_ITEMS; ++it) {
    if (q[it] == (real)0) continue;
    // fast path: all 2^d corners inside the window (the common case)
    int lc[D];
    bool fast = true;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      lc[m] = (c[it][m] - org[m]) & mask;
      fast &= lc[m] + 1 < ext[m];
    }
    if (fast) {
      const real qs = q[it] * scale;
      const real wx0 = (real)1 - f[it][0], wx1 = f[it][0];
      if (D == 2) {
        const int base = lc[0] + ext[0] * lc[1 % D];
        const real a = qs * ((real)1 - f[it][1 % D]), b = qs * f[it][1 % D];
        atomicAdd(&win[base], W::quantize_fma(a, wx0));
        atomicAdd(&win[base + 1], W::quantize_fma(a, wx1));
        atomicAdd(&win[base + ext[0]], W::quantize_fma(b, wx0));
        atomicAdd(&win[base + ext[0] + 1], W::quantize_fma(b, wx1));
      } else {
        const int sy = ext[0], sz = ext[0] * ext[1 % D];
        const int base = lc[0] + sy * lc[1 % D] + sz * lc[(D - 1)];
        const real wy[2] = {(real)1 - f[it][1 % D], f[it][1 % D]};
        const real wz[2] = {(real)1 - f[it][D - 1], f[it][D - 1]};
#pragma unroll
        for (int kz = 0; kz < 2; ++kz)
#pragma unroll
          for (int ky = 0; ky < 2; ++ky) {
            const real a = qs * wz[kz] * wy[ky];
            const int o = base + kz * sz + ky * sy;
            atomicAdd(&win[o], W::quantize_fma(a, wx0));
            atomicAdd(&win[o + 1], W::quantize_fma(a, wx1));
          }
      }
      continue;
    }
#pragma unroll
    for (int corner = 0; corner < (1 << D); ++corner) {
      real wgt = q[it];
      int loc = 0, glob = 0, lstride = 1, gstride = 1;
      bool inside = true;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        const int b = (corner >> m) & 1;
        wgt *= b ? f[it][m] : ((real)1 - f[it][m]);
        const int g = (c[it][m] + b) & mask;
        const int l = (g - org[m]) & mask;
        inside &= l < ext[m];
        loc += l * lstride;
        lstride *= ext[m];
        glob += g * gstride;
        gstride *= N;
      }
      if (inside) {
        atomicAdd(&win[loc], W::quantize_fma(wgt, scale));
      } else {
        atomicAdd(&rho[glob], wgt);
      }
    }
  }
  __syncthreads();
  // ---- flush: one warp per window row, lanes along x (coalesced atomics)
  const int rows = nwin / ext[0];
  for (int r = threadIdx.x >> 5; r < rows; r += DEP_THREADS / 32) {
    size_t grow;
    if (D == 2) {
      grow = (size_t)((org[1 % D] + r) & mask) * N;
    } else {
      const int ry = r % ext[1 % D], rz = r / ext[1 % D];
      grow = ((size_t)((org[D - 1] + rz) & mask) * N + ((org[1 % D] + ry) & mask)) * N;
    }
    const T* wrow = win + (size_t)r * ext[0];
    for (int x = lane; x < ext[0]; x += 32) {
      const T sv = wrow[x];
      if (sv != (T)0) atomicAdd(&rho[grow + ((org[0] + x) & mask)], W::value(sv, inv_scale));
    }
  }
}

template <typename real, int D>
int launch_deposit(const PArrays<real, D>& p, size_t np, int n, real inv_cell_vol, real* rho, int win_cap_nodes,
                   cudaStream_t s) {
  if (np == 0) return SG_OK;
  unsigned blocks = (unsigned)((np + DEP_CHUNK - 1) / DEP_CHUNK);
  using T = typename WinAcc<real>::T;
  const long long cap = (long long)win_cap_nodes * 8 / (long long)sizeof(T);  // same bytes for either type
  int side = 1;  // largest side with side^D <= capacity
  while (true) {
    long long nxt = 1;
    for (int m = 0; m < D; ++m) nxt *= (side + 1);
    if (nxt > cap) break;
    ++side;
  }
  long long nodes = 1;
  for (int m = 0; m < D; ++m) nodes *= side;
  const size_t smem = ((size_t)nodes * sizeof(T) + 15) / 16 * 16;  // zeroed in 16-byte words
  static bool attr_set = false;
  if (!attr_set) {
    if (smem > 48 * 1024)
      SG_CUDA(cudaFuncSetAttribute(k_deposit<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    SG_CUDA(cudaFuncSetAttribute(k_deposit<real, D>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr_set = true;
  }
  k_deposit<real, D><<<blocks, DEP_THREADS, smem, s>>>(p, np, n, inv_cell_vol, rho, side);
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

template <typename real, int VPL>
__global__ void __launch_bounds__(256) k_restrict_warp(const LineJob* __restrict__ jobs, int njobs) {
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
  const RjOut<real> e{J, o, i, lane};
  int level = top;
  const int tmin = J->tmin;
  if (VPL > 1 || top >= 5) {
    e.template emit<VPL>(v, level);
    if (level > tmin) RjLevels<real, VPL>::run(v, level, tmin, e);
  } else if (((J->tmask >> level) & 1) && lane < len) {  // a line shorter than a warp
    reinterpret_cast<real*>(J->dst[level])[((o << level) + lane) * (size_t)inner + i] = v[0];
  }
  // one value per lane on m = 2^level lanes
  real a = v[0];
  while (level > tmin) {
    const int m = 1 << level, h = m >> 1;
    const int k = lane & (h - 1);
    const real am = __shfl_sync(0xffffffffu, a, (2 * k - 1) & (m - 1));
    const real a0 = __shfl_sync(0xffffffffu, a, (2 * k) & (m - 1));
    const real ap = __shfl_sync(0xffffffffu, a, (2 * k + 1) & (m - 1));
    a = (real)0.25 * am + (real)0.5 * a0 + (real)0.25 * ap;
    --level;
    if (((J->tmask >> level) & 1) && lane < h)
      reinterpret_cast<real*>(J->dst[level])[((o << level) + lane) * (size_t)inner + i] = a;
  }
}

template <typename real>
int launch_restrict_pass(const LineJob* jobs_dev, int njobs, int nblocks, int lines_per_block, int vpl,
                         int smem_bytes, cudaStream_t s) {
  if (njobs == 0 || nblocks == 0) return SG_OK;
  const unsigned threads = 32u * (unsigned)lines_per_block;
#define SG_RJ_CASE(V)                                                                                     \
  case V: {                                                                                               \
    static bool attr_set = false;                                                                         \
    if (!attr_set) {                                                                                      \
      SG_CUDA(cudaFuncSetAttribute(k_restrict_warp<real, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   200 * 1024));                                                          \
      attr_set = true;                                                                                    \
    }                                                                                                     \
    SG_CUDA(launch_pdl(k_restrict_warp<real, V>, dim3(nblocks), dim3(threads), smem_bytes, s, jobs_dev, njobs)); \
    break;                                                                                                \
  }
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
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_DEP(real, D)                                                                            \
  template int launch_deposit<real, D>(const PArrays<real, D>&, size_t, int, real, real*, int, cudaStream_t);

SG_INST_DEP(float, 2)
SG_INST_DEP(float, 3)
SG_INST_DEP(double, 2)
SG_INST_DEP(double, 3)
template int launch_restrict_pass<float>(const LineJob*, int, int, int, int, int, cudaStream_t);
template int launch_restrict_pass<double>(const LineJob*, int, int, int, int, int, cudaStream_t);

}  // namespace sg
