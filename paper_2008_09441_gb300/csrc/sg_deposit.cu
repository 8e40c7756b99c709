// CIC charge deposition onto the regular level-n grid through a
// shared-memory window per particle chunk, and the restriction pyramid that
// carries the regular density to every component grid.
//
// Proposition 1 (Section 4.1, Appendix A): for node-centred grids and linear
// shapes, depositing on the regular grid and then applying R_i
// (eq. restriction) gives exactly the direct deposit onto component grid i.
// The GPU therefore deposits 2^d corners per particle once and restricts,
// instead of 2^d * n_c scattered adds per particle.
#include <limits.h>

#include "sg_kernels.cuh"

namespace sg {

// Shared-memory accumulator of the deposit window.  FP32 path: 32-bit fixed
// point (native integer shared atomics; a contribution is rounded once, to
// 2^-30 of the chunk's total |charge|, and integer sums are order-independent).
// FP64 path: plain double.
template <typename real>
struct WinAcc;
template <>
struct WinAcc<float> {
  using T = int;
  static constexpr int bits = 30;
  static __device__ __forceinline__ T quantize(float x) { return __float2int_rn(x); }
  static __device__ __forceinline__ float value(T s, float inv_scale) { return (float)s * inv_scale; }
};
template <>
struct WinAcc<double> {
  using T = double;
  static constexpr int bits = 0;
  static __device__ __forceinline__ T quantize(double x) { return x; }
  static __device__ __forceinline__ double value(T s, double) { return s; }
};

// ---------------------------------------------------------------- deposit
//
// Each block takes DEP_CHUNK consecutive particles (consecutive in tile-key
// order after a sort, so they occupy a compact block of cells).  All of them
// are loaded first (16-byte vector loads); the chunk's middle particle fixes
// the anchor cell and the periodic bounding box of the chunk's cells sizes a
// window of regular nodes in shared memory, accumulated with WinAcc (for
// the FP32 path the fixed-point scale is 2^30 / (sum of the chunk's |q_p| / V)
// rounded down to a power of two, so no node can overflow).  Non-zero window
// nodes are then added to the global grid in the run's precision.  Corners outside a window clamped to
// the shared-memory capacity add directly to the global grid.
template <typename real, int D>
__global__ void __launch_bounds__(DEP_THREADS) k_deposit(PArrays<real, D> p, size_t np, int n,
                                                         real inv_cell_vol, real* __restrict__ rho, int side) {
  extern __shared__ unsigned char smem_raw[];
  using W = WinAcc<real>;
  using T = typename W::T;
  T* win = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_anchor[D], s_min[D], s_max[D];
  __shared__ double s_wq[DEP_THREADS / 32];
  const int N = 1 << n;
  const int mask = N - 1;
  const size_t chunk = (size_t)blockIdx.x * DEP_CHUNK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

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
  double qabs = 0.0;
#pragma unroll
  for (int it = 0; it < DEP_ITEMS; ++it) {
    const size_t i = chunk + ((size_t)(it >> 2) * DEP_THREADS + threadIdx.x) * 4 + (it & 3);
    if (i < np) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        const real s = ub[it][m] * (real)N;
        int ci = (int)s;
        ci = ci < 0 ? 0 : (ci > mask ? mask : ci);
        c[it][m] = ci;
        f[it][m] = s - (real)ci;
        const int dd = ((ci - anchor[m] + (N >> 1)) & mask) - (N >> 1);
        dmin[m] = min(dmin[m], dd);
        dmax[m] = max(dmax[m], dd);
      }
      q[it] = wb[it] * inv_cell_vol;
      qabs += fabs((double)q[it]);
    } else {
      q[it] = (real)0;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        c[it][m] = anchor[m];
        f[it][m] = (real)0;
      }
    }
  }
  qabs = warp_sum(qabs);
  if (lane == 0) s_wq[warp] = qabs;
#pragma unroll
  for (int m = 0; m < D; ++m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmin[m] = min(dmin[m], __shfl_xor_sync(0xffffffffu, dmin[m], o));
      dmax[m] = max(dmax[m], __shfl_xor_sync(0xffffffffu, dmax[m], o));
    }
    if (lane == 0) {
      atomicMin(&s_min[m], dmin[m]);
      atomicMax(&s_max[m], dmax[m]);
    }
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
  double qsum = 0.0;
#pragma unroll
  for (int w = 0; w < DEP_THREADS / 32; ++w) qsum += s_wq[w];
  int ex = 0;
  frexp(qsum, &ex);  // qsum < 2^ex
  const bool fixed = W::bits > 0 && qsum > 0.0;
  const real scale = fixed ? (real)ldexp(1.0, W::bits - ex) : (real)1;
  const real inv_scale = fixed ? (real)ldexp(1.0, ex - W::bits) : (real)1;
  for (int i = threadIdx.x; i < nwin; i += DEP_THREADS) win[i] = (T)0;
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
      const real w0[2] = {(real)1 - f[it][0], f[it][0]};
      if (D == 2) {
        const int base = lc[0] + ext[0] * lc[1];
        const real a = qs * ((real)1 - f[it][1]), b = qs * f[it][1];
        atomicAdd(&win[base], W::quantize(a * w0[0]));
        atomicAdd(&win[base + 1], W::quantize(a * w0[1]));
        atomicAdd(&win[base + ext[0]], W::quantize(b * w0[0]));
        atomicAdd(&win[base + ext[0] + 1], W::quantize(b * w0[1]));
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
            atomicAdd(&win[o], W::quantize(a * w0[0]));
            atomicAdd(&win[o + 1], W::quantize(a * w0[1]));
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
        atomicAdd(&win[loc], W::quantize(wgt * scale));
      } else {
        atomicAdd(&rho[glob], wgt);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nwin; i += DEP_THREADS) {
    const T sv = win[i];
    if (sv != (T)0) {
      int rem = i, glob = 0, gstride = 1;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        const int l = rem % ext[m];
        rem /= ext[m];
        glob += ((org[m] + l) & mask) * gstride;
        gstride *= N;
      }
      atomicAdd(&rho[glob], W::value(sv, inv_scale));
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
  size_t smem = (size_t)nodes * sizeof(T);
  static bool attr_set = false;
  if (smem > 48 * 1024 && !attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_deposit<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_deposit<real, D><<<blocks, DEP_THREADS, smem, s>>>(p, np, n, inv_cell_vol, rho, side);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// ---------------------------------------------------------------- restriction pyramid
//
// A line of length 2^top along `axis` is restricted level by level:
// b[k] = (a[2k-1] + 2 a[2k] + a[2k+1]) / 4 (periodic), which is
// (h_l / h_{l-1}) sum_k' W_{l-1}(x_k - x_k') a[k'] -- the one-axis R of
// eq. restriction from level l to l-1.  Composing the steps is exact because
// a coarse hat is linear between the finer nodes (Appendix A).
template <typename real>
__global__ void __launch_bounds__(256) k_restrict_lines(const LineJob* __restrict__ jobs, int njobs) {
  extern __shared__ unsigned char smem_raw[];
  real* buf = reinterpret_cast<real*>(smem_raw);
  int b = blockIdx.x;
  const int j = find_job(jobs, njobs);
  const LineJob& J = jobs[j];
  const int top = J.top;
  const int len = 1 << top;
  const int C = J.lines_per_block;
  const int line0 = (b - J.block_begin) * C;
  // All extents are powers of two and lines_per_block divides the line
  // count, so index arithmetic is shifts and masks.
  const int nl = C;
  const int logC = __ffs(C) - 1;
  int ls = 0;  // log2 of the stride of the line axis
  for (int m = 0; m < J.axis; ++m) ls += __ffs(J.dims[m]) - 1;
  const long long smask = (1ll << ls) - 1;
  const real* src = reinterpret_cast<const real*>(J.src);
  // levels as a heap: level l of line li at [li * 2 len + 2^l, li * 2 len + 2^(l+1))
  const int slot = 2 * len;
  for (int e = threadIdx.x; e < (nl << top); e += blockDim.x) {
    int li, t;
    if (J.axis == 0) {
      li = e >> top;
      t = e & (len - 1);
    } else {  // consecutive threads take consecutive lines (coalesced columns)
      li = e & (nl - 1);
      t = e >> logC;
    }
    const long long L = line0 + li;
    const long long addr = (L & smask) + (((long long)t + ((L >> ls) << top)) << ls);
    buf[li * slot + len + t] = src[addr];
  }
  __syncthreads();
  for (int l = top - 1; l >= 0; --l) {
    const int cnt = 1 << l;
    const int up = 1 << (l + 1);  // size of the finer level
    for (int e = threadIdx.x; e < (nl << l); e += blockDim.x) {
      const int li = e >> l, k = e & (cnt - 1);
      const real* a = buf + li * slot + up;
      const real am = a[(2 * k - 1 + up) & (up - 1)];
      const real a0 = a[2 * k];
      const real ap = a[(2 * k + 1) & (up - 1)];
      buf[li * slot + cnt + k] = (real)0.25 * am + (real)0.5 * a0 + (real)0.25 * ap;
    }
    __syncthreads();
  }
  for (int tg = 0; tg < J.ntargets; ++tg) {
    const int tl = J.tlev[tg];
    const int tlen = 1 << tl;
    real* dst = reinterpret_cast<real*>(J.dst[tg]);
    for (int e = threadIdx.x; e < (nl << tl); e += blockDim.x) {
      int li, t;
      if (J.axis == 0) {
        li = e >> tl;
        t = e & (tlen - 1);
      } else {
        li = e & (nl - 1);
        t = e >> logC;
      }
      const long long L = line0 + li;
      const long long addr = (L & smask) + (((long long)t + ((L >> ls) << tl)) << ls);
      dst[addr] = buf[li * slot + tlen + t];
    }
  }
}

template <typename real>
int launch_restrict_pass(const LineJob* jobs_dev, int njobs, int nblocks, int smem_bytes, cudaStream_t s) {
  if (njobs == 0 || nblocks == 0) return SG_OK;
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_restrict_lines<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_restrict_lines<real><<<nblocks, 256, smem_bytes, s>>>(jobs_dev, njobs);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_DEP(real, D)                                                                            \
  template int launch_deposit<real, D>(const PArrays<real, D>&, size_t, int, real, real*, int, cudaStream_t);

SG_INST_DEP(float, 2)
SG_INST_DEP(float, 3)
SG_INST_DEP(double, 2)
SG_INST_DEP(double, 3)
template int launch_restrict_pass<float>(const LineJob*, int, int, int, cudaStream_t);
template int launch_restrict_pass<double>(const LineJob*, int, int, int, cudaStream_t);

}  // namespace sg
