// Batched spectral Poisson solves over all component grids (Section 2:
// -Laplace phi = rho, E = -grad phi; spectral discretisation).
//
// Each grid's 2D/3D transform is split into passes of 1D radix-2 FFTs along
// one axis; one launch per pass covers every line of every component grid
// (of every resident run when batched).  A block stages a few lines in
// shared memory, transforms them with an iterative decimation-in-time FFT
// (bit-reversed load, natural-order result) and writes them back.  The last
// forward axis is fused with the spectral multiply
//   phi^ = rho^ / |k|^2 (k = 0 -> 0),  E^_m = -i k_m phi^ (Nyquist of axis m -> 0)
// and the first inverse axis of every field component.
#include "sg_kernels.cuh"

namespace sg {

template <typename real>
__device__ __forceinline__ void fft_smem(cplx<real>* buf, int nl, int logn, bool inverse,
                                         const cplx<real>* __restrict__ tw, int log_nmax) {
  const int len = 1 << logn;
  const int halfN = len >> 1;
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    const int tshift = log_nmax - s;
    for (int j = threadIdx.x; j < nl * halfN; j += blockDim.x) {
      int li = j >> (logn - 1);
      int jj = j & (halfN - 1);
      int pos = jj & (half - 1);
      int grp = jj >> (s - 1);
      int i0 = li * len + grp * 2 * half + pos;
      int i1 = i0 + half;
      cplx<real> w = tw[pos << tshift];
      if (inverse) w.y = -w.y;
      cplx<real> a = buf[i0], b = buf[i1];
      real bx = b.x * w.x - b.y * w.y;
      real by = b.x * w.y + b.y * w.x;
      buf[i0] = {a.x + bx, a.y + by};
      buf[i1] = {a.x - bx, a.y - by};
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int t, int logn) { return logn == 0 ? 0 : (int)(__brev((unsigned)t) >> (32 - logn)); }

// element (line li of the block, position t) -> array offset, for lines along
// `axis` of an array with dims; consecutive threads take consecutive lines
// when axis > 0 so that strided columns are read together.
__device__ __forceinline__ long long line_addr(long long L, int t, long long stride, int len) {
  long long low = L % stride, high = L / stride;
  return low + stride * ((long long)t + (long long)len * high);
}

__device__ __forceinline__ int sfreq(int i, int N) { return i < (N >> 1) ? i : i - N; }

template <typename real>
__global__ void __launch_bounds__(256) k_fft_pass(int kind, SolveArena<real> a, const FftJob* __restrict__ jobs,
                                                  int njobs) {
  extern __shared__ unsigned char smem_raw[];
  int b = blockIdx.x;
  const int j = find_job(jobs, njobs);
  const FftJob& J = jobs[j];
  const GridDesc g = a.grids[J.grid];
  const int logn = J.logn;
  const int len = 1 << logn;
  const int C = J.lines_per_block;
  const int line0 = (b - J.block_begin) * C;
  const int nl = min(C, J.lines - line0);
  if (nl <= 0) return;
  cplx<real>* buf0 = reinterpret_cast<cplx<real>*>(smem_raw);
  cplx<real>* buf1 = buf0 + C * len;
  long long stride = 1;
  for (int m = 0; m < J.axis; ++m) stride *= J.dims[m];
  const size_t S = a.S;
  const bool contiguous = (J.axis == 0);

  // load
  for (int e = threadIdx.x; e < nl * len; e += blockDim.x) {
    int li = contiguous ? e / len : e % nl;
    int t = contiguous ? e % len : e / nl;
    long long off = line_addr(line0 + li, t, stride, len);
    cplx<real> v;
    if (kind == FFT_FWD_FIRST) {
      v.x = a.rho[g.offset + off];
      v.y = (real)0;
    } else if (kind == FFT_FWD_MID || kind == FFT_LAST) {
      v = a.A[g.offset + off];
    } else {
      v = a.B[(size_t)J.comp * S + g.offset + off];
    }
    buf0[li * len + bitrev(t, logn)] = v;
  }
  __syncthreads();
  const bool inverse = (kind == FFT_INV_MID || kind == FFT_INV_LAST);
  fft_smem<real>(buf0, nl, logn, inverse, a.tw, a.log_nmax);

  if (kind == FFT_LAST) {
    const int D = a.dim;
    const real norm = (real)1 / (real)g.size;
    for (int m = 0; m < D; ++m) {
      for (int e = threadIdx.x; e < nl * len; e += blockDim.x) {
        int li = e / len, t = e % len;
        long long L = line0 + li;  // combined index of the axes before the last
        int idx[3];
        idx[D - 1] = t;
        if (D == 2) {
          idx[0] = (int)L;
        } else {
          idx[0] = (int)(L % J.dims[0]);
          idx[1] = (int)(L / J.dims[0]);
        }
        real k2 = 0, km = 0;
        bool nyq_m = false;
        for (int q = 0; q < D; ++q) {
          int Nq = J.dims[q];
          real kq = (real)(g.kfac[q] * (double)sfreq(idx[q], Nq));
          k2 += kq * kq;
          if (q == m) {
            km = kq;
            nyq_m = (idx[q] == (Nq >> 1));
          }
        }
        cplx<real> r = buf0[li * len + t];
        cplx<real> out;
        if (k2 == (real)0 || nyq_m) {
          out = {(real)0, (real)0};
        } else {
          real fac = km / k2 * norm;  // -i k_m rho^/|k|^2 : (a + ib) -> (b, -a)
          out = {r.y * fac, -r.x * fac};
        }
        buf1[li * len + bitrev(t, logn)] = out;
      }
      __syncthreads();
      fft_smem<real>(buf1, nl, logn, true, a.tw, a.log_nmax);
      for (int e = threadIdx.x; e < nl * len; e += blockDim.x) {
        int li = contiguous ? e / len : e % nl;
        int t = contiguous ? e % len : e / nl;
        long long off = line_addr(line0 + li, t, stride, len);
        a.B[(size_t)m * S + g.offset + off] = buf1[li * len + t];
      }
      __syncthreads();
    }
    return;
  }

  for (int e = threadIdx.x; e < nl * len; e += blockDim.x) {
    int li = contiguous ? e / len : e % nl;
    int t = contiguous ? e % len : e / nl;
    long long off = line_addr(line0 + li, t, stride, len);
    cplx<real> v = buf0[li * len + t];
    if (kind == FFT_FWD_FIRST || kind == FFT_FWD_MID) {
      a.A[g.offset + off] = v;
    } else if (kind == FFT_INV_MID) {
      a.B[(size_t)J.comp * S + g.offset + off] = v;
    } else {  // FFT_INV_LAST: the field is real
      a.E[(size_t)J.comp * S + g.offset + off] = v.x;
    }
  }
}

template <typename real>
int launch_fft_pass(int kind, const SolveArena<real>& a, const FftJob* jobs_dev, int njobs, int nblocks,
                    int smem_bytes, cudaStream_t s) {
  if (njobs == 0 || nblocks == 0) return SG_OK;
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_fft_pass<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_fft_pass<real><<<nblocks, 256, smem_bytes, s>>>(kind, a, jobs_dev, njobs);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// ---------------------------------------------------------------- one block per grid
//
// When every component grid fits in shared memory (twice: spectrum and one
// field component), one launch solves all of them: a block loads its grid,
// transforms it along every axis in place (bit-reversal swap, then the
// butterfly stages), forms each E^_m and transforms it back.
template <typename real>
__device__ void fft_axis_inplace(cplx<real>* buf, const int* dims, const int* logs, int S, int ax, bool inverse,
                                 const cplx<real>* __restrict__ tw, int log_nmax) {
  const int len = dims[ax], logn = logs[ax];
  int stride = 1;
  for (int m = 0; m < ax; ++m) stride *= dims[m];
  for (int e = threadIdx.x; e < S; e += blockDim.x) {
    const int t = (e / stride) & (len - 1);
    const int r = bitrev(t, logn);
    if (r > t) {
      const int e2 = e + (r - t) * stride;
      cplx<real> x = buf[e];
      buf[e] = buf[e2];
      buf[e2] = x;
    }
  }
  __syncthreads();
  const int halfN = len >> 1;
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    const int tshift = log_nmax - s;
    for (int j = threadIdx.x; j < (S >> 1); j += blockDim.x) {
      const int L = j >> (logn - 1);
      const int jj = j & (halfN - 1);
      const int pos = jj & (half - 1);
      const int grp = jj >> (s - 1);
      const int t0 = grp * 2 * half + pos;
      const int low = L % stride, high = L / stride;
      const int i0 = low + stride * (t0 + len * high);
      const int i1 = i0 + half * stride;
      cplx<real> w = tw[pos << tshift];
      if (inverse) w.y = -w.y;
      cplx<real> x0 = buf[i0], x1 = buf[i1];
      real bx = x1.x * w.x - x1.y * w.y;
      real by = x1.x * w.y + x1.y * w.x;
      buf[i0] = {x0.x + bx, x0.y + by};
      buf[i1] = {x0.x - bx, x0.y - by};
    }
    __syncthreads();
  }
}

template <typename real>
__global__ void __launch_bounds__(1024) k_solve_small(SolveArena<real> a) {
  extern __shared__ unsigned char smem_raw[];
  const GridDesc g = a.grids[blockIdx.x];
  const int D = a.dim;
  int dims[3] = {1, 1, 1}, logs[3] = {0, 0, 0};
  for (int m = 0; m < D; ++m) {
    logs[m] = g.l[m];
    dims[m] = 1 << g.l[m];
  }
  const int S = g.size;
  cplx<real>* A = reinterpret_cast<cplx<real>*>(smem_raw);
  cplx<real>* B = A + S;
  for (int e = threadIdx.x; e < S; e += blockDim.x) A[e] = {a.rho[g.offset + e], (real)0};
  __syncthreads();
  for (int ax = 0; ax < D; ++ax) fft_axis_inplace<real>(A, dims, logs, S, ax, false, a.tw, a.log_nmax);
  const real norm = (real)1 / (real)S;
  for (int m = 0; m < D; ++m) {
    for (int e = threadIdx.x; e < S; e += blockDim.x) {
      int idx[3];
      idx[0] = e & (dims[0] - 1);
      idx[1] = (e >> logs[0]) & (dims[1] - 1);
      idx[2] = D == 3 ? (e >> (logs[0] + logs[1])) : 0;
      real k2 = 0, km = 0;
      bool nyq_m = false;
      for (int q = 0; q < D; ++q) {
        const real kq = (real)(g.kfac[q] * (double)sfreq(idx[q], dims[q]));
        k2 += kq * kq;
        if (q == m) {
          km = kq;
          nyq_m = idx[q] == (dims[q] >> 1);
        }
      }
      const cplx<real> r = A[e];
      if (k2 == (real)0 || nyq_m) {
        B[e] = {(real)0, (real)0};
      } else {
        const real fac = km / k2 * norm;
        B[e] = {r.y * fac, -r.x * fac};
      }
    }
    __syncthreads();
    for (int ax = 0; ax < D; ++ax) fft_axis_inplace<real>(B, dims, logs, S, ax, true, a.tw, a.log_nmax);
    for (int e = threadIdx.x; e < S; e += blockDim.x) a.E[(size_t)m * a.S + g.offset + e] = B[e].x;
    __syncthreads();
  }
}

template <typename real>
int launch_solve_small(const SolveArena<real>& a, int ngrids, int max_size, cudaStream_t s) {
  if (ngrids == 0) return SG_OK;
  int threads = max_size / 2;
  threads = threads < 64 ? 64 : (threads > 1024 ? 1024 : threads);
  size_t smem = (size_t)2 * max_size * sizeof(cplx<real>);
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_solve_small<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_solve_small<real><<<ngrids, threads, smem, s>>>(a);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template int launch_solve_small<float>(const SolveArena<float>&, int, int, cudaStream_t);
template int launch_solve_small<double>(const SolveArena<double>&, int, int, cudaStream_t);

// In-place FFT of a whole N^D complex array along one axis (regular grid).
template <typename real>
__global__ void __launch_bounds__(256) k_fft_array(cplx<real>* data, int D, int logn, int axis, int inverse,
                                                   const cplx<real>* __restrict__ tw, int log_nmax, int C) {
  extern __shared__ unsigned char smem_raw[];
  cplx<real>* buf = reinterpret_cast<cplx<real>*>(smem_raw);
  const int len = 1 << logn;
  long long lines = 1;
  for (int m = 0; m < D - 1; ++m) lines *= len;
  long long line0 = (long long)blockIdx.x * C;
  int nl = (int)min((long long)C, lines - line0);
  if (nl <= 0) return;
  long long stride = 1;
  for (int m = 0; m < axis; ++m) stride *= len;
  const bool contiguous = axis == 0;
  for (int e = threadIdx.x; e < nl * len; e += blockDim.x) {
    int li = contiguous ? e / len : e % nl;
    int t = contiguous ? e % len : e / nl;
    buf[li * len + bitrev(t, logn)] = data[line_addr(line0 + li, t, stride, len)];
  }
  __syncthreads();
  fft_smem<real>(buf, nl, logn, inverse != 0, tw, log_nmax);
  for (int e = threadIdx.x; e < nl * len; e += blockDim.x) {
    int li = contiguous ? e / len : e % nl;
    int t = contiguous ? e % len : e / nl;
    data[line_addr(line0 + li, t, stride, len)] = buf[li * len + t];
  }
}

template <typename real>
int launch_fft_array_axis(cplx<real>* data, int D, int logn, int axis, bool inverse, const cplx<real>* tw,
                          int log_nmax, cudaStream_t s) {
  const int len = 1 << logn;
  int C = 2048 / len;
  if (C < 1) C = 1;
  if (axis > 0 && C < 8) C = 8;  // wider column blocks for coalescing
  long long lines = 1;
  for (int m = 0; m < D - 1; ++m) lines *= len;
  if (C > lines) C = (int)lines;
  size_t smem = (size_t)C * len * sizeof(cplx<real>);
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_fft_array<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  unsigned blocks = (unsigned)((lines + C - 1) / C);
  k_fft_array<real><<<blocks, 256, smem, s>>>(data, D, logn, axis, inverse ? 1 : 0, tw, log_nmax, C);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template int launch_fft_pass<float>(int, const SolveArena<float>&, const FftJob*, int, int, int, cudaStream_t);
template int launch_fft_pass<double>(int, const SolveArena<double>&, const FftJob*, int, int, int, cudaStream_t);
template int launch_fft_array_axis<float>(cplx<float>*, int, int, int, bool, const cplx<float>*, int, cudaStream_t);
template int launch_fft_array_axis<double>(cplx<double>*, int, int, int, bool, const cplx<double>*, int,
                                           cudaStream_t);

}  // namespace sg
