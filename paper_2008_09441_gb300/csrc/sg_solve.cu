// Batched spectral Poisson solves over all component grids (Section 2:
// -Laplace phi = rho, E = -grad phi; spectral discretisation).
//
// Each grid's 2D/3D transform is split into passes of 1D radix-2 FFTs along
// one axis; one launch per pass covers every line of every component grid
// of the run.  A block stages a few lines in
// shared memory, transforms them with an iterative decimation-in-time FFT
// (bit-reversed load, natural-order result) and writes them back.  The last
// forward axis is fused with the spectral multiply
//   phi^ = rho^ / |k|^2 (k = 0 -> 0),  E^_m = -i k_m phi^ (Nyquist of axis m -> 0)
// and the first inverse axis of every field component.
#include "sg_kernels.cuh"

namespace sg {

template <typename real>
__device__ __forceinline__ cplx<real> cmul(cplx<real> a, cplx<real> w) {
  return {a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x};
}

// Iterative decimation-in-time FFT of nl lines of length 2^logn in shared
// memory (input in bit-reversed order, output natural).  Stages are taken in
// pairs (radix 2^2): a thread loads four elements {i, i+h, i+2h, i+3h}, does
// the two butterflies of stage s (span 2h) and the two of stage s+1 (span
// 4h) in registers and stores them, halving the passes over shared memory and
// the barriers; an odd last stage is a plain radix-2 pass.
// Shared-memory index of element x of the line buffers: one padding element
// after every 32, so that the bit-reversed stores (consecutive t land 2^(logn-5)
// apart) and the large-span butterflies spread over the banks.
__device__ __forceinline__ int fpad(int x) { return x + (x >> 5); }
__host__ __device__ constexpr size_t fpad_size(size_t n) { return n + (n >> 5); }

// Twiddles are stage-major (twiddle_index): the lanes of a warp read
// consecutive entries in every stage, free of bank conflicts.
template <typename real>
__device__ __forceinline__ void fft_smem(cplx<real>* buf, int nl, int logn, bool inverse,
                                         const cplx<real>* __restrict__ tw) {
  const int len = 1 << logn;
  const int halfN = len >> 1;
  int s0 = 1;
  for (; s0 + 1 <= logn; s0 += 2) {
    const int h = 1 << (s0 - 1);
    const int quarter = len >> 2;
    for (int j = threadIdx.x; j < nl * quarter; j += blockDim.x) {
      const int li = j >> (logn - 2);
      const int jj = j & (quarter - 1);
      const int pos = jj & (h - 1);
      const int grp = jj >> (s0 - 1);
      const int i0 = li * len + grp * 4 * h + pos;
      // W_{2h}^pos, W_{4h}^pos and W_{4h}^(pos + h)
      cplx<real> w1 = tw[twiddle_index(h, pos)], w2 = tw[twiddle_index(2 * h, pos)],
                 w3 = tw[twiddle_index(2 * h, pos + h)];
      if (inverse) {
        w1.y = -w1.y;
        w2.y = -w2.y;
        w3.y = -w3.y;
      }
      const cplx<real> a0 = buf[fpad(i0)], a1 = buf[fpad(i0 + h)], a2 = buf[fpad(i0 + 2 * h)],
                       a3 = buf[fpad(i0 + 3 * h)];
      const cplx<real> m1 = cmul(a1, w1), m3 = cmul(a3, w1);
      const cplx<real> b0 = {a0.x + m1.x, a0.y + m1.y}, b1 = {a0.x - m1.x, a0.y - m1.y};
      const cplx<real> b2 = {a2.x + m3.x, a2.y + m3.y}, b3 = {a2.x - m3.x, a2.y - m3.y};
      const cplx<real> n2 = cmul(b2, w2), n3 = cmul(b3, w3);
      buf[fpad(i0)] = {b0.x + n2.x, b0.y + n2.y};
      buf[fpad(i0 + 2 * h)] = {b0.x - n2.x, b0.y - n2.y};
      buf[fpad(i0 + h)] = {b1.x + n3.x, b1.y + n3.y};
      buf[fpad(i0 + 3 * h)] = {b1.x - n3.x, b1.y - n3.y};
    }
    __syncthreads();
  }
  for (int s = s0; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    for (int j = threadIdx.x; j < nl * halfN; j += blockDim.x) {
      int li = j >> (logn - 1);
      int jj = j & (halfN - 1);
      int pos = jj & (half - 1);
      int grp = jj >> (s - 1);
      int i0 = li * len + grp * 2 * half + pos;
      int i1 = i0 + half;
      cplx<real> w = tw[twiddle_index(half, pos)];
      if (inverse) w.y = -w.y;
      cplx<real> a = buf[fpad(i0)], b = buf[fpad(i1)];
      real bx = b.x * w.x - b.y * w.y;
      real by = b.x * w.y + b.y * w.x;
      buf[fpad(i0)] = {a.x + bx, a.y + by};
      buf[fpad(i1)] = {a.x - bx, a.y - by};
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int t, int logn) { return logn == 0 ? 0 : (int)(__brev((unsigned)t) >> (32 - logn)); }

// element (line L, position t) -> array offset for lines along an axis whose
// stride is 2^ls in an array of power-of-two extents (line length 2^logn).
__device__ __forceinline__ long long line_addr(long long L, int t, int ls, int logn) {
  return (L & ((1ll << ls) - 1)) + (((long long)t + ((L >> ls) << logn)) << ls);
}

__device__ __forceinline__ int sfreq(int i, int N) { return i < (N >> 1) ? i : i - N; }

// Lines per block (C) are a power of two dividing the line count; for lines
// along axis > 0 consecutive threads take consecutive lines so that strided
// columns are read together.
template <typename real>
__global__ void __launch_bounds__(FFT_BLOCK_VALUES / 2) k_fft_pass(int kind, SolveArena<real> a, const FftJob* __restrict__ jobs,
                                                  int njobs) {
  extern __shared__ unsigned char smem_raw[];
  const int b = blockIdx.x;
  pdl_trigger();
  const int j = find_job(jobs, njobs);  // job and grid tables are written once, at set-up
  const FftJob& J = jobs[j];
  const GridDesc g = a.grids[J.grid];
  const int logn = J.logn;
  const int len = 1 << logn;
  const int C = J.lines_per_block;
  const int logC = __ffs(C) - 1;
  const int line0 = (b - J.block_begin) * C;
  const int nl = C;
  // twiddles staged in shared memory, then the two line buffers
  cplx<real>* tws = reinterpret_cast<cplx<real>*>(smem_raw);
  const int ntw = twiddle_count(a.log_nmax);
  for (int e = threadIdx.x; e < ntw; e += blockDim.x) tws[e] = a.tw[e];
  pdl_wait();  // the previous pass's output
  cplx<real>* buf0 = tws + ntw;
  cplx<real>* buf1 = buf0 + fpad_size((size_t)C * len);
  int ls = 0;
  for (int m = 0; m < J.axis; ++m) ls += __ffs(J.dims[m]) - 1;
  const size_t S = a.S;
  const bool contiguous = (J.axis == 0);
  const int total = nl << logn;

  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int li = contiguous ? (e >> logn) : (e & (nl - 1));
    const int t = contiguous ? (e & (len - 1)) : (e >> logC);
    const long long off = line_addr(line0 + li, t, ls, logn);
    cplx<real> v;
    if (kind == FFT_FWD_FIRST) {
      v.x = a.rho[g.offset + off];
      v.y = (real)0;
    } else if (kind == FFT_FWD_MID || kind == FFT_LAST) {
      v = a.A[g.offset + off];
    } else {
      v = a.B[(size_t)J.comp * S + g.offset + off];
    }
    buf0[fpad((li << logn) + bitrev(t, logn))] = v;
  }
  __syncthreads();
  const bool inverse = (kind == FFT_INV_MID || kind == FFT_INV_LAST);
  fft_smem<real>(buf0, nl, logn, inverse, tws);

  if (kind == FFT_LAST) {
    const int D = a.dim;
    const real norm = (real)1 / (real)g.size;
    const int l0 = __ffs(J.dims[0]) - 1;
    for (int p = 0; 2 * p < D; ++p) {
      const int ma = 2 * p, mb = 2 * p + 1;  // mb == D: no second component
      for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int li = e >> logn, t = e & (len - 1);
        const int L = line0 + li;  // combined index of the axes before the last
        int idx[3];
        idx[D - 1] = t;
        if (D == 2) {
          idx[0] = L;
        } else {
          idx[0] = L & (J.dims[0] - 1);
          idx[1] = L >> l0;
        }
        real k2 = 0, ka = 0, kb = 0;
        bool nyq_a = false, nyq_b = false;
        for (int q = 0; q < D; ++q) {
          const int Nq = J.dims[q];
          const real kq = (real)g.kfac[q] * (real)sfreq(idx[q], Nq);  // no FP64 on the FP32 path
          k2 += kq * kq;
          if (q == ma) {
            ka = kq;
            nyq_a = (idx[q] == (Nq >> 1));
          }
          if (q == mb) {
            kb = kq;
            nyq_b = (idx[q] == (Nq >> 1));
          }
        }
        const cplx<real> r = buf0[fpad((li << logn) + t)];
        // E^_m = -i k_m rho^ / |k|^2 : (x + iy) -> (y, -x) * k_m / |k|^2
        cplx<real> out = {(real)0, (real)0};
        if (k2 != (real)0) {
          const real inv = norm / k2;
          if (!nyq_a) {
            const real fa = ka * inv;
            out.x += r.y * fa;
            out.y -= r.x * fa;
          }
          if (mb < D && !nyq_b) {  // + i E^_b: (y, -x) * fb times i -> (x, y) * fb
            const real fb = kb * inv;
            out.x += r.x * fb;
            out.y += r.y * fb;
          }
        }
        buf1[fpad((li << logn) + bitrev(t, logn))] = out;
      }
      __syncthreads();
      fft_smem<real>(buf1, nl, logn, true, tws);
      for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int li = contiguous ? (e >> logn) : (e & (nl - 1));
        const int t = contiguous ? (e & (len - 1)) : (e >> logC);
        const long long off = line_addr(line0 + li, t, ls, logn);
        a.B[(size_t)p * S + g.offset + off] = buf1[fpad((li << logn) + t)];
      }
      __syncthreads();
    }
    return;
  }

  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int li = contiguous ? (e >> logn) : (e & (nl - 1));
    const int t = contiguous ? (e & (len - 1)) : (e >> logC);
    const long long off = line_addr(line0 + li, t, ls, logn);
    const cplx<real> v = buf0[fpad((li << logn) + t)];
    if (kind == FFT_FWD_FIRST || kind == FFT_FWD_MID) {
      a.A[g.offset + off] = v;
    } else if (kind == FFT_INV_MID) {
      a.B[(size_t)J.comp * S + g.offset + off] = v;
    } else {  // FFT_INV_LAST: real part -> component 2p, imaginary -> 2p + 1
      a.E[(size_t)(2 * J.comp) * S + g.offset + off] = v.x;
      if (2 * J.comp + 1 < a.dim) a.E[(size_t)(2 * J.comp + 1) * S + g.offset + off] = v.y;
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
  SG_CUDA(launch_pdl(k_fft_pass<real>, dim3(nblocks), dim3(FFT_BLOCK_VALUES / 2),
                     smem_bytes + (size_t)twiddle_count(a.log_nmax) * sizeof(cplx<real>), s, kind, a, jobs_dev,
                     njobs));
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
__device__ void fft_axis_inplace(cplx<real>* buf, const int* logs, int S, int ax, bool inverse,
                                 const cplx<real>* __restrict__ tw) {
  const int logn = logs[ax];
  const int len = 1 << logn;
  int ls = 0;
  for (int m = 0; m < ax; ++m) ls += logs[m];
  const int smask = (1 << ls) - 1;
  for (int e = threadIdx.x; e < S; e += blockDim.x) {
    const int t = (e >> ls) & (len - 1);
    const int r = bitrev(t, logn);
    if (r > t) {
      const int e2 = e + ((r - t) << ls);
      cplx<real> x = buf[e];
      buf[e] = buf[e2];
      buf[e2] = x;
    }
  }
  __syncthreads();
  const int halfN = len >> 1;
  // Butterfly j of a stage: consecutive j take consecutive inner indices
  // (the axes below ax, contiguous in the buffer), then the butterflies of
  // one line, then the outer lines, so that a warp's accesses are
  // contiguous along every axis (the line itself strides by 2^ls).
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    for (int j = threadIdx.x; j < (S >> 1); j += blockDim.x) {
      const int i = j & smask;
      const int p = (j >> ls) & (halfN - 1);
      const int o = j >> (ls + logn - 1);
      const int pos = p & (half - 1);
      const int grp = p >> (s - 1);
      const int t0 = grp * 2 * half + pos;
      const int i0 = (((o << logn) + t0) << ls) + i;
      const int i1 = i0 + (half << ls);
      cplx<real> w = tw[twiddle_index(half, pos)];
      if (inverse) w.y = -w.y;
      const cplx<real> x0 = buf[i0], x1 = buf[i1];
      const real bx = x1.x * w.x - x1.y * w.y;
      const real by = x1.x * w.y + x1.y * w.x;
      buf[i0] = {x0.x + bx, x0.y + by};
      buf[i1] = {x0.x - bx, x0.y - by};
    }
    __syncthreads();
  }
}

// One block solves grid gi of arena a: load, forward transforms, E^_m,
// paired inverse transforms, store.
template <typename real>
__device__ __forceinline__ void solve_grid_block(const SolveArena<real>& a, int gi, int max_size) {
  extern __shared__ unsigned char smem_raw[];
  const GridDesc g = a.grids[gi];
  const int D = a.dim;
  int logs[3] = {0, 0, 0};
  for (int m = 0; m < D; ++m) logs[m] = g.l[m];
  const int S = g.size;
  cplx<real>* A = reinterpret_cast<cplx<real>*>(smem_raw);
  cplx<real>* B = A + max_size;
  cplx<real>* tws = B + max_size;  // twiddle table staged in shared memory
  const int ntw = twiddle_count(a.log_nmax);
  for (int e = threadIdx.x; e < ntw; e += blockDim.x) tws[e] = a.tw[e];
  for (int e = threadIdx.x; e < S; e += blockDim.x) A[e] = {a.rho[g.offset + e], (real)0};
  __syncthreads();
  for (int ax = 0; ax < D; ++ax) fft_axis_inplace<real>(A, logs, S, ax, false, tws);
  const real norm = (real)1 / (real)S;
  const int n0 = 1 << logs[0], n1 = 1 << logs[1];
  // Field components in pairs: B = E^_a + i E^_b, one inverse transform,
  // E_a its real part and E_b its imaginary part (both fields are real).
  for (int pr = 0; 2 * pr < D; ++pr) {
    const int ma = 2 * pr, mb = 2 * pr + 1;
    for (int e = threadIdx.x; e < S; e += blockDim.x) {
      int idx[3];
      idx[0] = e & (n0 - 1);
      idx[1] = (e >> logs[0]) & (n1 - 1);
      idx[2] = D == 3 ? (e >> (logs[0] + logs[1])) : 0;
      real k2 = 0, ka = 0, kb = 0;
      bool nyq_a = false, nyq_b = false;
      for (int q = 0; q < D; ++q) {
        const int Nq = 1 << logs[q];
        const real kq = (real)g.kfac[q] * (real)sfreq(idx[q], Nq);
        k2 += kq * kq;
        if (q == ma) {
          ka = kq;
          nyq_a = idx[q] == (Nq >> 1);
        }
        if (q == mb) {
          kb = kq;
          nyq_b = idx[q] == (Nq >> 1);
        }
      }
      const cplx<real> r = A[e];
      cplx<real> out = {(real)0, (real)0};
      if (k2 != (real)0) {
        const real inv = norm / k2;
        if (!nyq_a) {  // E^_a = -i k_a rho^ / |k|^2
          const real fa = ka * inv;
          out.x += r.y * fa;
          out.y -= r.x * fa;
        }
        if (mb < D && !nyq_b) {  // + i E^_b
          const real fb = kb * inv;
          out.x += r.x * fb;
          out.y += r.y * fb;
        }
      }
      B[e] = out;
    }
    __syncthreads();
    for (int ax = 0; ax < D; ++ax) fft_axis_inplace<real>(B, logs, S, ax, true, tws);
    for (int e = threadIdx.x; e < S; e += blockDim.x) {
      a.E[(size_t)ma * a.S + g.offset + e] = B[e].x;
      if (mb < D) a.E[(size_t)mb * a.S + g.offset + e] = B[e].y;
    }
    __syncthreads();
  }
}

template <typename real>
__global__ void __launch_bounds__(1024) k_solve_small(SolveArena<real> a, int max_size, int grid0) {
  solve_grid_block<real>(a, grid0 + blockIdx.x, max_size);
}

// The cross-run solve: block b takes job b, a grid of one of the runs.
template <typename real>
__global__ void __launch_bounds__(1024) k_solve_batch(const SolveJob<real>* __restrict__ jobs, int max_size) {
  const SolveJob<real>& J = jobs[blockIdx.x];
  const SolveArena<real> a = J.a;
  solve_grid_block<real>(a, J.grid, max_size);
}

template <typename real>
int launch_solve_small(const SolveArena<real>& a, int ngrids, int max_size, cudaStream_t s, int grid0) {
  if (ngrids == 0) return SG_OK;
  int threads = max_size / 2;
  threads = threads < 64 ? 64 : (threads > 1024 ? 1024 : threads);
  size_t smem = ((size_t)2 * max_size + (size_t)twiddle_count(a.log_nmax)) * sizeof(cplx<real>);
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_solve_small<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_solve_small<real><<<ngrids, threads, smem, s>>>(a, max_size, grid0);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template int launch_solve_small<float>(const SolveArena<float>&, int, int, cudaStream_t, int);
template int launch_solve_small<double>(const SolveArena<double>&, int, int, cudaStream_t, int);

template <typename real>
int launch_solve_batch(const SolveJob<real>* jobs, int njobs, int max_size, int max_log, cudaStream_t s) {
  if (njobs == 0) return SG_OK;
  if (max_size > small_solve_max<real>()) {
    set_error("cross-run solve: a component grid is larger than one block's shared memory takes");
    return SG_ERR_UNSUPPORTED;
  }
  int threads = max_size / 2;
  threads = threads < 64 ? 64 : (threads > 1024 ? 1024 : threads);
  const size_t smem = ((size_t)2 * max_size + (size_t)twiddle_count(max_log)) * sizeof(cplx<real>);
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_solve_batch<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_solve_batch<real><<<njobs, threads, smem, s>>>(jobs, max_size);
  SG_CHECK_LAUNCH();
  return SG_OK;
}
template int launch_solve_batch<float>(const SolveJob<float>*, int, int, int, cudaStream_t);
template int launch_solve_batch<double>(const SolveJob<double>*, int, int, int, cudaStream_t);

// In-place FFT of a whole N^D complex array along one axis (regular grid).
template <typename real>
__global__ void __launch_bounds__(256) k_fft_array(cplx<real>* data, int D, int logn, int axis, int inverse,
                                                   const cplx<real>* __restrict__ tw, int log_nmax, int C) {
  extern __shared__ unsigned char smem_raw[];
  // twiddles staged in shared memory, then the lines
  cplx<real>* tws = reinterpret_cast<cplx<real>*>(smem_raw);
  const int ntw = twiddle_count(log_nmax);
  for (int e = threadIdx.x; e < ntw; e += blockDim.x) tws[e] = tw[e];
  cplx<real>* buf = tws + ntw;
  const int len = 1 << logn;
  const long long line0 = (long long)blockIdx.x * C;  // C is a power of two dividing the line count
  const int nl = C;
  const int logC = __ffs(C) - 1;
  const int ls = axis * logn;
  const bool contiguous = axis == 0;
  for (int e = threadIdx.x; e < (nl << logn); e += blockDim.x) {
    const int li = contiguous ? (e >> logn) : (e & (nl - 1));
    const int t = contiguous ? (e & (len - 1)) : (e >> logC);
    buf[fpad((li << logn) + bitrev(t, logn))] = data[line_addr(line0 + li, t, ls, logn)];
  }
  __syncthreads();
  fft_smem<real>(buf, nl, logn, inverse != 0, tws);
  for (int e = threadIdx.x; e < (nl << logn); e += blockDim.x) {
    const int li = contiguous ? (e >> logn) : (e & (nl - 1));
    const int t = contiguous ? (e & (len - 1)) : (e >> logC);
    data[line_addr(line0 + li, t, ls, logn)] = buf[fpad((li << logn) + t)];
  }
}

template <typename real>
int launch_fft_array_axis(cplx<real>* data, int D, int logn, int axis, bool inverse, const cplx<real>* tw,
                          int log_nmax, cudaStream_t s) {
  const int len = 1 << logn;
  int C = 2048 / len;
  if (C < 1) C = 1;
  if (axis > 0 && C < 4) C = 4;  // column blocks: 32-byte row pieces (complex float), more blocks than SMs
  long long lines = 1;
  for (int m = 0; m < D - 1; ++m) lines *= len;
  if (C > lines) C = (int)lines;
  size_t smem = (fpad_size((size_t)C * len) + (size_t)twiddle_count(log_nmax)) * sizeof(cplx<real>);
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

// ---------------------------------------------------------------- filter mode: the regular-grid solve
//
// Algorithm 2's field step on the 2^{dn} regular nodes: F(rho_f) (a complex
// copy transformed along every axis), then per pair of field components
// B = E^_a + i E^_b with E^_m = -i k_m rho^ / |k|^2 (k = 0 and the Nyquist
// plane of axis m -> 0, the component-grid rules), the inverse transform
// along every axis, and the real / imaginary parts as E_a / E_b.

template <typename real>
__global__ void k_regular_pack(const real* __restrict__ rho, cplx<real>* __restrict__ a, size_t nd) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += (size_t)gridDim.x * blockDim.x)
    a[i] = {rho[i], (real)0};
}

// ktab[m * N + i] = 2 pi / L_m * (i < N/2 ? i : i - N), in the run's precision.
template <typename real>
__global__ void k_regular_spectral(const cplx<real>* __restrict__ A, cplx<real>* __restrict__ B, int dim, int n,
                                   const real* __restrict__ ktab, int pair, real norm) {
  const int N = 1 << n, mask = N - 1;
  const size_t nd = (size_t)1 << (dim * n);
  const int ma = 2 * pair, mb = 2 * pair + 1;  // mb == dim: no second component
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += (size_t)gridDim.x * blockDim.x) {
    real k2 = 0, ka = 0, kb = 0;
    bool nyq_a = false, nyq_b = false;
    for (int q = 0; q < dim; ++q) {
      const int idx = (int)(i >> (q * n)) & mask;
      const real kq = ktab[q * N + idx];
      k2 += kq * kq;
      if (q == ma) {
        ka = kq;
        nyq_a = idx == (N >> 1);
      }
      if (q == mb) {
        kb = kq;
        nyq_b = idx == (N >> 1);
      }
    }
    const cplx<real> r = A[i];
    cplx<real> out = {(real)0, (real)0};
    if (k2 != (real)0) {
      const real inv = norm / k2;
      if (!nyq_a) {  // -i k_a rho^ / |k|^2
        const real fa = ka * inv;
        out.x += r.y * fa;
        out.y -= r.x * fa;
      }
      if (mb < dim && !nyq_b) {  // + i (-i k_b rho^ / |k|^2)
        const real fb = kb * inv;
        out.x += r.x * fb;
        out.y += r.y * fb;
      }
    }
    B[i] = out;
  }
}

// E_hi[node * stride + 2p (+1)] from the pair's inverse transform; the FP32
// path's low planes of these components are zero.  Per-block partials of
// sum |E|^2 at partials[pair * gridDim.x + block].
template <typename real>
__global__ void __launch_bounds__(256) k_regular_field_out(const cplx<real>* __restrict__ B, real* __restrict__ Ehi,
                                                           float* __restrict__ Elo, int dim, int stride, size_t nd,
                                                           int pair, double* __restrict__ partials) {
  __shared__ double red[32];
  const int ma = 2 * pair, mb = 2 * pair + 1;
  real energy = (real)0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += (size_t)gridDim.x * blockDim.x) {
    const cplx<real> v = B[i];
    Ehi[i * stride + ma] = v.x;
    energy = fma(v.x, v.x, energy);
    if (Elo) Elo[(size_t)ma * nd + i] = 0.f;
    if (mb < dim) {
      Ehi[i * stride + mb] = v.y;
      energy = fma(v.y, v.y, energy);
      if (Elo) Elo[(size_t)mb * nd + i] = 0.f;
    }
  }
  const double tot = block_sum_double((double)energy, red);
  if (threadIdx.x == 0) partials[(size_t)pair * gridDim.x + blockIdx.x] = tot;
}

template <typename real>
int launch_regular_solve(const real* rho_f, cplx<real>* A, cplx<real>* B, const real* ktab,
                         const cplx<real>* tw, int dim, int n, real* Ehi, float* Elo, int stride, double* partials,
                         int blocks, cudaStream_t s) {
  const size_t nd = (size_t)1 << (dim * n);
  k_regular_pack<real><<<blocks, 256, 0, s>>>(rho_f, A, nd);
  SG_CHECK_LAUNCH();
  for (int ax = 0; ax < dim; ++ax) SG_TRY(launch_fft_array_axis<real>(A, dim, n, ax, false, tw, n, s));
  const real norm = (real)(1.0 / (double)nd);
  for (int p = 0; 2 * p < dim; ++p) {
    k_regular_spectral<real><<<blocks, 256, 0, s>>>(A, B, dim, n, ktab, p, norm);
    SG_CHECK_LAUNCH();
    for (int ax = 0; ax < dim; ++ax) SG_TRY(launch_fft_array_axis<real>(B, dim, n, ax, true, tw, n, s));
    k_regular_field_out<real><<<blocks, 256, 0, s>>>(B, Ehi, Elo, dim, stride, nd, p, partials);
    SG_CHECK_LAUNCH();
  }
  return SG_OK;
}
template int launch_regular_solve<float>(const float*, cplx<float>*, cplx<float>*, const float*,
                                         const cplx<float>*, int, int, float*, float*, int, double*, int,
                                         cudaStream_t);
template int launch_regular_solve<double>(const double*, cplx<double>*, cplx<double>*, const double*,
                                          const cplx<double>*, int, int, double*, float*, int, double*, int,
                                          cudaStream_t);

template int launch_fft_pass<float>(int, const SolveArena<float>&, const FftJob*, int, int, int, cudaStream_t);
template int launch_fft_pass<double>(int, const SolveArena<double>&, const FftJob*, int, int, int, cudaStream_t);
template int launch_fft_array_axis<float>(cplx<float>*, int, int, int, bool, const cplx<float>*, int, cudaStream_t);
template int launch_fft_array_axis<double>(cplx<double>*, int, int, int, bool, const cplx<double>*, int,
                                           cudaStream_t);

}  // namespace sg
