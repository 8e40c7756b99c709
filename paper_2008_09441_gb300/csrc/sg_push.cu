// Gather + push (Section 2, steps 3-4): CIC interpolation of the combined
// field (same shape as the deposit) plus the linear external field, then a
// leapfrog kick (Boris rotation when B != 0) and the drift
// x^{n+1} = x^n + v^{n+1/2} dt, wrapped into the periodic box.  Each thread
// also adds 0.5 m_p v^{n-1/2}.v^{n+1/2} to the time-centred kinetic energy.
#include "sg_kernels.cuh"

namespace sg {

static __device__ __forceinline__ bool finite_r(float x) { return isfinite(x); }
static __device__ __forceinline__ bool finite_r(double x) { return isfinite(x); }

int push_blocks(size_t np) {
  size_t b = (np + 255) / 256;
  const size_t cap = 152 * 16;
  if (b > cap) b = cap;
  if (b == 0) b = 1;
  return (int)b;
}

template <typename real, int D>
__global__ void __launch_bounds__(256) k_push(PArrays<real, D> p, size_t np, int n, const real* __restrict__ Ec,
                                              PushParams<real> pp, double* __restrict__ ke_partials,
                                              unsigned* status) {
  __shared__ double red[32];
  const int N = 1 << n;
  const int mask = N - 1;
  const size_t ND = (size_t)N * (D == 2 ? N : (size_t)N * N);
  const real half = (real)0.5;
  Acc<real> ke;
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
    real u[D], v[D], E[D];
    int c[D];
    real f[D];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      u[m] = p.u[m][i];
      v[m] = p.v[m][i];
      real s = u[m] * (real)N;
      int ci = (int)s;
      ci = ci < 0 ? 0 : (ci > mask ? mask : ci);
      c[m] = ci;
      f[m] = s - (real)ci;
      E[m] = (real)0;
    }
    const real w = p.w[i];
#pragma unroll
    for (int corner = 0; corner < (1 << D); ++corner) {
      real wgt = (real)1;
      size_t node = 0, gs = 1;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        int b = (corner >> m) & 1;
        wgt *= b ? f[m] : ((real)1 - f[m]);
        node += (size_t)((c[m] + b) & mask) * gs;
        gs *= (size_t)N;
      }
#pragma unroll
      for (int m = 0; m < D; ++m) E[m] += wgt * __ldg(Ec + (size_t)m * ND + node);
    }
    if (pp.has_eext) {
#pragma unroll
      for (int m = 0; m < D; ++m) E[m] += pp.eext[m] * (u[m] - half);
    }
    real vm[D], vn[D];
    const real hk = pp.qm * pp.dt * half;
#pragma unroll
    for (int m = 0; m < D; ++m) vm[m] = v[m] + hk * E[m];
    if (pp.boris) {
      if (D == 2) {
        const real tz = pp.tB[2];
        const real sz = (real)2 * tz / ((real)1 + tz * tz);
        const real px = vm[0] + vm[1] * tz;
        const real py = vm[1] - vm[0] * tz;
        vm[0] = vm[0] + py * sz;
        vm[1] = vm[1] - px * sz;
      } else {
        const real t0 = pp.tB[0], t1 = pp.tB[1], t2 = pp.tB[2];
        const real tt = t0 * t0 + t1 * t1 + t2 * t2;
        const real s0 = (real)2 * t0 / ((real)1 + tt), s1 = (real)2 * t1 / ((real)1 + tt),
                   s2 = (real)2 * t2 / ((real)1 + tt);
        const real a0 = vm[D > 1 ? 0 : 0], a1 = vm[1], a2 = vm[D - 1];
        const real p0 = a0 + (a1 * t2 - a2 * t1);
        const real p1 = a1 + (a2 * t0 - a0 * t2);
        const real p2 = a2 + (a0 * t1 - a1 * t0);
        vm[0] = a0 + (p1 * s2 - p2 * s1);
        vm[1] = a1 + (p2 * s0 - p0 * s2);
        vm[D - 1] = a2 + (p0 * s1 - p1 * s0);
      }
    }
    real dot = (real)0;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      vn[m] = vm[m] + hk * E[m];
      dot += v[m] * vn[m];
      bad |= !finite_r(vn[m]);
      p.v[m][i] = vn[m];
    }
    ke.add(half * (w / pp.qm) * dot);
    if (pp.drift) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        real un = wrap_unit(u[m] + vn[m] * pp.dt_over_L[m]);
        bad |= !finite_r(un);
        p.u[m][i] = un;
      }
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
  double tot = block_sum_double(ke.to_double(), red);
  if (threadIdx.x == 0 && ke_partials) ke_partials[blockIdx.x] = tot;
}

template <typename real, int D>
int launch_push(const PArrays<real, D>& p, size_t np, int n, const real* Ecomb, PushParams<real> pp,
                double* ke_partials, unsigned* status, cudaStream_t s) {
  int blocks = push_blocks(np);
  k_push<real, D><<<blocks, 256, 0, s>>>(p, np, n, Ecomb, pp, ke_partials, status);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_PUSH(real, D)                                                                           \
  template int launch_push<real, D>(const PArrays<real, D>&, size_t, int, const real*, PushParams<real>, \
                                    double*, unsigned*, cudaStream_t);
SG_INST_PUSH(float, 2)
SG_INST_PUSH(float, 3)
SG_INST_PUSH(double, 2)
SG_INST_PUSH(double, 3)

}  // namespace sg
