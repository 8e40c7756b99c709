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

// ---------------------------------------------------------------- deposit
//
// Each block takes DEP_CHUNK consecutive particles (consecutive in the
// cell-key order after a sort, so they occupy a compact Morton block).  It
// sizes a window of regular nodes around them (periodic displacement from
// the chunk's middle particle), accumulates the CIC weights in shared memory
// and adds the non-zero window nodes to the global grid.  Particles whose
// corners fall outside a window clamped to the shared-memory capacity add
// directly to the global grid.
template <typename real, int D>
__global__ void __launch_bounds__(DEP_THREADS) k_deposit(PArrays<real, D> p, size_t np, int n,
                                                         real inv_cell_vol, real* __restrict__ rho,
                                                         int win_cap) {
  extern __shared__ unsigned char smem_raw[];
  real* win = reinterpret_cast<real*>(smem_raw);
  __shared__ int s_anchor[D], s_min[D], s_max[D], s_org[D], s_ext[D];
  __shared__ int s_nwin;
  const int N = 1 << n;
  const int mask = N - 1;
  const size_t chunk = (size_t)blockIdx.x * DEP_CHUNK;
  if (threadIdx.x == 0) {
    size_t mid = chunk + DEP_CHUNK / 2;
    if (mid >= np) mid = np - 1;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      s_anchor[m] = cell_of(p.u[m][mid], n, N);
      s_min[m] = INT_MAX;
      s_max[m] = INT_MIN;
    }
  }
  __syncthreads();

  int c[DEP_ITEMS][D];
  real f[DEP_ITEMS][D];
  real q[DEP_ITEMS];
  int dmin[D], dmax[D];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    dmin[m] = INT_MAX;
    dmax[m] = INT_MIN;
  }
  // Items: DEP_ITEMS / 4 vectors of four consecutive particles per thread
  // (16-byte loads); the ragged end of the last chunk is read element-wise.
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
#pragma unroll
  for (int it = 0; it < DEP_ITEMS; ++it) {
    const size_t i = chunk + ((size_t)(it >> 2) * DEP_THREADS + threadIdx.x) * 4 + (it & 3);
    if (i < np) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        real s = ub[it][m] * (real)N;
        int ci = (int)s;
        ci = ci < 0 ? 0 : (ci > mask ? mask : ci);
        c[it][m] = ci;
        f[it][m] = s - (real)ci;
        int dd = ((ci - s_anchor[m] + (N >> 1)) & mask) - (N >> 1);
        dmin[m] = min(dmin[m], dd);
        dmax[m] = max(dmax[m], dd);
      }
      q[it] = wb[it] * inv_cell_vol;
    } else {
      q[it] = (real)0;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        c[it][m] = s_anchor[m];
        f[it][m] = (real)0;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < D; ++m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmin[m] = min(dmin[m], __shfl_xor_sync(0xffffffffu, dmin[m], o));
      dmax[m] = max(dmax[m], __shfl_xor_sync(0xffffffffu, dmax[m], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&s_min[m], dmin[m]);
      atomicMax(&s_max[m], dmax[m]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int side = 1;
    while (true) {  // largest side with side^D <= win_cap
      long long nxt = 1;
      for (int m = 0; m < D; ++m) nxt *= (side + 1);
      if (nxt > win_cap) break;
      ++side;
    }
    long long nw = 1;
    for (int m = 0; m < D; ++m) {
      int lo = s_min[m], ext;
      if (lo == INT_MAX) {  // empty chunk (cannot happen for launched blocks)
        lo = 0;
        ext = 1;
      } else {
        ext = s_max[m] - lo + 2;  // +1 node for the upper corner
      }
      if (ext >= N) {  // the window spans the whole axis
        ext = N;
        lo = -(N >> 1);
      }
      if (ext > side) {  // clamp around the anchor; outliers add to global
        ext = side;
        lo = -(side >> 1);
      }
      s_org[m] = (s_anchor[m] + lo) & mask;
      s_ext[m] = ext;
      nw *= ext;
    }
    s_nwin = (int)nw;
  }
  __syncthreads();
  const int nwin = s_nwin;
  for (int i = threadIdx.x; i < nwin; i += DEP_THREADS) win[i] = (real)0;
  int org[D], ext[D];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    org[m] = s_org[m];
    ext[m] = s_ext[m];
  }
  __syncthreads();

#pragma unroll
  for (int it = 0; it < DEP_ITEMS; ++it) {
    if (q[it] == (real)0) continue;
#pragma unroll
    for (int corner = 0; corner < (1 << D); ++corner) {
      real wgt = q[it];
      int loc = 0, glob = 0, lstride = 1, gstride = 1;
      bool inside = true;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        int b = (corner >> m) & 1;
        wgt *= b ? f[it][m] : ((real)1 - f[it][m]);
        int g = (c[it][m] + b) & mask;
        int l = (g - org[m]) & mask;
        inside &= l < ext[m];
        loc += l * lstride;
        lstride *= ext[m];
        glob += g * gstride;
        gstride *= N;
      }
      if (inside)
        atomicAdd(&win[loc], wgt);
      else
        atomicAdd(&rho[glob], wgt);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nwin; i += DEP_THREADS) {
    real val = win[i];
    if (val != (real)0) {
      int rem = i, glob = 0, gstride = 1;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        int l = rem % ext[m];
        rem /= ext[m];
        glob += ((org[m] + l) & mask) * gstride;
        gstride *= N;
      }
      atomicAdd(&rho[glob], val);
    }
  }
}

template <typename real, int D>
int launch_deposit(const PArrays<real, D>& p, size_t np, int n, real inv_cell_vol, real* rho, int win_cap_nodes,
                   cudaStream_t s) {
  if (np == 0) return SG_OK;
  unsigned blocks = (unsigned)((np + DEP_CHUNK - 1) / DEP_CHUNK);
  size_t smem = (size_t)win_cap_nodes * sizeof(real);
  static bool attr_set = false;
  if (smem > 48 * 1024 && !attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_deposit<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_deposit<real, D><<<blocks, DEP_THREADS, smem, s>>>(p, np, n, inv_cell_vol, rho, win_cap_nodes);
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
