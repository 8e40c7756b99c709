// FP64 diagnostics reductions, conversions and the device halves of the
// tauEstimator (Algorithm 1): thresholding and spectral-derivative products
// of the regular-grid density's Fourier coefficients, and max-norms.
#include <cstring>

#include "sg_kernels.cuh"

namespace sg {

static __device__ __forceinline__ bool finite_r(float x) { return isfinite(x); }
static __device__ __forceinline__ bool finite_r(double x) { return isfinite(x); }

// Wrap positions into [0,1) and flag non-finite particle data (run init).
template <typename real, int D>
__global__ void k_wrap_check(PArrays<real, D> p, size_t np, unsigned* status) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  bool bad = !finite_r(p.w[i]);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    real u = p.u[m][i];
    bad |= !finite_r(u) || !finite_r(p.v[m][i]);
    if (finite_r(u)) p.u[m][i] = wrap_unit(u);
  }
  p.pid[i] = (uint32_t)i;
  if (bad) atomicOr(status, ST_NONFINITE);
}

template <typename real, int D>
int launch_wrap_check(const PArrays<real, D>& p, size_t np, unsigned* status, cudaStream_t s) {
  if (np == 0) return SG_OK;
  k_wrap_check<real, D><<<(unsigned)((np + 255) / 256), 256, 0, s>>>(p, np, status);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// The upload's statistics in one pass: per block the FP64 sum of the charges
// (grid-stride over the particles, then the block) at out[b], the largest
// |q| at out[nb + b], and the status word of the upload check at
// out[2 nb] (as its bits).
template <typename real>
__global__ void k_charge_stats(const real* w, size_t n, const unsigned* status, double* out) {
  __shared__ double red[32];
  __shared__ double wmax[32];
  double acc = 0.0, mx = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double q = (double)w[i];
    acc += q;
    mx = fmax(mx, fabs(q));
  }
  const double t = block_sum_double(acc, red);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, wmax[k]);
    out[blockIdx.x] = t;
    out[gridDim.x + blockIdx.x] = m;
    if (blockIdx.x == 0) {
      unsigned long long st = *status;
      out[2 * gridDim.x] = __longlong_as_double((long long)st);
    }
  }
}

template <typename real>
int launch_charge_stats(const real* w, size_t n, const unsigned* status, double* out, int nblocks, cudaStream_t s) {
  k_charge_stats<real><<<nblocks, 256, 0, s>>>(w, n, status, out);
  SG_CHECK_LAUNCH();
  return SG_OK;
}
template int launch_charge_stats<float>(const float*, size_t, const unsigned*, double*, int, cudaStream_t);
template int launch_charge_stats<double>(const double*, size_t, const unsigned*, double*, int, cudaStream_t);

// End-of-step bookkeeping: field energy of the new combined field, the
// previous one, and the kinetic energy of the push, all FP64.
__global__ void k_finalize_step(const double* fe_partials, int n_fe, const double* ke_partials, int n_ke,
                                double fe_scale, DevDiag* dd) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n_fe; i += blockDim.x) a += fe_partials[i];
  double fe = block_sum_double(a, red);
  double b = 0.0;
  if (ke_partials)
    for (int i = threadIdx.x; i < n_ke; i += blockDim.x) b += ke_partials[i];
  double ke = block_sum_double(b, red);
  if (threadIdx.x == 0) {
    dd->field_energy_prev = dd->field_energy;
    dd->field_energy = fe * fe_scale;
    if (ke_partials) dd->kinetic_energy = ke;
  }
}

int launch_finalize_step(const double* fe_partials, int n_fe, const double* ke_partials, int n_ke,
                         double fe_scale, DevDiag* dd, cudaStream_t s) {
  k_finalize_step<<<1, 1024, 0, s>>>(fe_partials, n_fe, ke_partials, n_ke, fe_scale, dd);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// The diagnostics record: the device record, the checksum, the status word
// and V_i sum_k rho_i(x_k) of every component grid's stored density, in
// FP64.  The grids hold deviations from the mean density: the host adds the
// mean's charge to obtain each grid's charge.
template <typename real>
__global__ void k_diag_record(const GridDesc* grids, const real* rho, const DevDiag* dd,
                              const unsigned long long* cks, const unsigned* st, unsigned char* out, size_t o_cks,
                              size_t o_ch) {
  __shared__ double red[32];
  const GridDesc g = grids[blockIdx.x];
  double acc = 0.0;
  for (int k = threadIdx.x; k < g.size; k += blockDim.x) acc += (double)rho[g.offset + k];
  const double t = block_sum_double(acc, red);
  if (threadIdx.x == 0) {
    reinterpret_cast<double*>(out + o_ch)[blockIdx.x] = t * g.vol;
    if (blockIdx.x == 0) {
      *reinterpret_cast<DevDiag*>(out) = *dd;
      *reinterpret_cast<unsigned long long*>(out + o_cks) = *cks;
      *reinterpret_cast<unsigned*>(out + o_cks + 8) = *st;
    }
  }
}

template <typename real>
int launch_diag_record(const GridDesc* grids, int ngrids, const real* rho, const DevDiag* dd,
                       const unsigned long long* cks, const unsigned* st, void* out, size_t o_cks, size_t o_ch,
                       cudaStream_t s) {
  if (ngrids < 1) return SG_OK;
  k_diag_record<real><<<ngrids, 256, 0, s>>>(grids, rho, dd, cks, st, static_cast<unsigned char*>(out), o_cks,
                                              o_ch);
  SG_CHECK_LAUNCH();
  return SG_OK;
}
template int launch_diag_record<float>(const GridDesc*, int, const float*, const DevDiag*, const unsigned long long*,
                                       const unsigned*, void*, size_t, size_t, cudaStream_t);
template int launch_diag_record<double>(const GridDesc*, int, const double*, const DevDiag*,
                                        const unsigned long long*, const unsigned*, void*, size_t, size_t,
                                        cudaStream_t);

template <typename real>
__global__ void k_to_double(const real* src, double* dst, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

template <typename real>
int launch_to_double(const real* src, double* dst, size_t n, cudaStream_t s) {
  if (n == 0) return SG_OK;
  k_to_double<real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template <typename real>
__global__ void k_field_to_double(const real* hi, const float* lo, double* dst, size_t nd, int dim, int stride) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd * (size_t)dim) return;
  const size_t m = i / nd, node = i - m * nd;
  dst[i] = (double)hi[node * (size_t)stride + m] + (lo ? (double)lo[i] : 0.0);
}

template <typename real>
int launch_field_to_double(const real* hi, const float* lo, double* dst, size_t nd, int dim, int stride,
                           cudaStream_t s) {
  const size_t n = nd * (size_t)dim;
  if (n == 0) return SG_OK;
  k_field_to_double<real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(hi, lo, dst, nd, dim, stride);
  SG_CHECK_LAUNCH();
  return SG_OK;
}
template int launch_field_to_double<float>(const float*, const float*, double*, size_t, int, int, cudaStream_t);
template int launch_field_to_double<double>(const double*, const float*, double*, size_t, int, int, cudaStream_t);

// max |x| through the float bits' order (non-negative values)
// ---------------------------------------------------------------- Algorithm 1 helpers (FP64)
__global__ void k_real_to_cplx(const double* src, cplx<double>* dst, size_t n, double scale) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = {src[i] * scale, 0.0};
}

int launch_real_to_cplx(const double* src, cplx<double>* dst, size_t n, double scale, cudaStream_t s) {
  k_real_to_cplx<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n, scale);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// Max of non-negative doubles via the order-preserving integer view.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <typename F>
__device__ __forceinline__ void block_max_store(double v, double* out) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomic_max_nonneg(out, v);
  }
}

struct MaxAbsC {};
__global__ void k_maxabs_cplx(const cplx<double>* z, size_t n, double* out) {
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, hypot(z[i].x, z[i].y));
  block_max_store<MaxAbsC>(m, out);
}

__global__ void k_maxabs_re(const cplx<double>* z, size_t n, double* out) {
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(z[i].x));
  block_max_store<MaxAbsC>(m, out);
}

__global__ void k_maxabs_real(const double* x, size_t n, double* out) {
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  block_max_store<MaxAbsC>(m, out);
}

static unsigned red_blocks(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b > 1216 ? 1216 : (b == 0 ? 1 : b));
}

int launch_maxabs_cplx(const cplx<double>* z, size_t n, double* out, cudaStream_t s) {
  SG_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  k_maxabs_cplx<<<red_blocks(n), 256, 0, s>>>(z, n, out);
  SG_CHECK_LAUNCH();
  return SG_OK;
}
int launch_maxabs_real_part(const cplx<double>* z, size_t n, double* out, cudaStream_t s) {
  SG_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  k_maxabs_re<<<red_blocks(n), 256, 0, s>>>(z, n, out);
  SG_CHECK_LAUNCH();
  return SG_OK;
}
int launch_maxabs_real(const double* x, size_t n, double* out, cudaStream_t s) {
  SG_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  k_maxabs_real<<<red_blocks(n), 256, 0, s>>>(x, n, out);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// eq. denoising: keep a mode if |rho^| >= eps, eps = frac * max|rho^|.
__global__ void k_threshold(cplx<double>* z, size_t n, const double* maxabs, double frac) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double eps = frac * (*maxabs);
  cplx<double> v = z[i];
  if (!(hypot(v.x, v.y) >= eps)) z[i] = {0.0, 0.0};
}

int launch_threshold(cplx<double>* z, size_t n, const double* maxabs, double frac, cudaStream_t s) {
  k_threshold<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(z, n, maxabs, frac);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// prod over the axes in `mask` of k_m^2 for DFT index i of an N^D array.
__device__ __forceinline__ double kprod(size_t i, int D, int logn, const double* kfac, int mask) {
  const int N = 1 << logn;
  double r = 1.0;
  for (int m = 0; m < D; ++m) {
    int im = (int)((i >> (m * logn)) & (size_t)(N - 1));
    if (mask & (1 << m)) {
      int f = im < (N >> 1) ? im : im - N;
      double k = kfac[m] * (double)f;
      r *= k * k;
    }
  }
  return r;
}

struct KF {
  double k[3];
};

__global__ void k_kmult(const cplx<double>* src, cplx<double>* dst, int D, int logn, KF kf, int mask, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = kprod(i, D, logn, kf.k, mask);
  dst[i] = {src[i].x * r, src[i].y * r};
}

int launch_kmult(const cplx<double>* src, cplx<double>* dst, int D, int logn, const double* kfac, int mask,
                 cudaStream_t s) {
  size_t n = (size_t)1 << (D * logn);
  KF kf{{kfac[0], kfac[1], D > 2 ? kfac[2] : 0.0}};
  k_kmult<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, D, logn, kf, mask, n);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

__global__ void k_maxabs_kmult(const cplx<double>* src, int D, int logn, KF kf, int mask, size_t n, double* out) {
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double r = kprod(i, D, logn, kf.k, mask);
    m = fmax(m, hypot(src[i].x * r, src[i].y * r));
  }
  block_max_store<MaxAbsC>(m, out);
}

int launch_maxabs_kmult(const cplx<double>* src, int D, int logn, const double* kfac, int mask, double* out,
                        cudaStream_t s) {
  size_t n = (size_t)1 << (D * logn);
  KF kf{{kfac[0], kfac[1], D > 2 ? kfac[2] : 0.0}};
  SG_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  k_maxabs_kmult<<<red_blocks(n), 256, 0, s>>>(src, D, logn, kf, mask, n, out);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_DIAG(real, D) template int launch_wrap_check<real, D>(const PArrays<real, D>&, size_t, unsigned*, cudaStream_t);
SG_INST_DIAG(float, 2)
SG_INST_DIAG(float, 3)
SG_INST_DIAG(double, 2)
SG_INST_DIAG(double, 3)
template int launch_to_double<float>(const float*, double*, size_t, cudaStream_t);
template int launch_to_double<double>(const double*, double*, size_t, cudaStream_t);

}  // namespace sg
