// Signed combination of the component fields on the regular nodes:
//   E_comb(x_j) = sum_i c_i (P_i E_i)(x_j)
// (eq. sparse_filter's c_i and P_i of eq. restriction, applied to the
// fields).  One block per regular row (a y line in 2D, a (y, z) line in
// 3D).  Every (level l, coarse x index k) pair of the row is an independent
// work item: it interpolates, in the transverse axes, every grid whose x level
// is l at the row's coordinate and adds c_i times the result (grids in a fixed
// order).  The x-prolongation is then applied once per level by Horner's
// scheme (prolong level l to l+1, add level l+1, ...), exact for nested
// node-centred grids.  Accumulation is float-float (FP32 path) or double
// (FP64 path); the row is written as hi / lo planes and contributes its share
// of sum |E_comb|^2 to the field energy.
#include "sg_kernels.cuh"

namespace sg {

template <typename real, int D>
__global__ void __launch_bounds__(256) k_combine(const GridDesc* __restrict__ grids, LevelLists ll, int lmin,
                                                 const real* __restrict__ E, size_t S, int n, real* __restrict__ Ehi,
                                                 float* __restrict__ Elo, double* __restrict__ partials,
                                                 const CombineFinal fin) {
  extern __shared__ unsigned char smem_raw[];
  Acc<real>* A = reinterpret_cast<Acc<real>*>(smem_raw);  // [D][2N], level l of comp m at m*2N + [2^l, 2^(l+1))
  __shared__ double red[32];
  const int N = 1 << n;
  const size_t ND = (size_t)N * (D == 2 ? N : (size_t)N * N);
  const int row = blockIdx.x;
  const int y = row & (N - 1);
  const int z = (D == 3) ? (row >> n) : 0;
  // Per-grid row parameters of this block's (y, z), computed once: the
  // 2^(d-1) coarse x-lines that bracket the row and their interpolation
  // weights (dyadic, exact), the grid's coefficient, in level-list order.
  constexpr int R = 1 << (D - 1);
  __shared__ int s_start[18];
  __shared__ int s_off[CB_MAX_GRIDS][R];
  __shared__ real s_w[CB_MAX_GRIDS][R];
  __shared__ real s_c[CB_MAX_GRIDS];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 18; ++i) s_start[i] = ll.start[i];  // constant indices: no local copy
  }
  const int ngl = ll.start[17];
  for (int gi = threadIdx.x; gi < ngl; gi += blockDim.x) {
    const GridDesc g = grids[ll.grid[gi]];
    const int nx = 1 << g.l[0];
    const int ry = n - g.l[1];
    const int ny = 1 << g.l[1];
    const int ky0 = y >> ry;
    const int ky1 = (ky0 + 1) & (ny - 1);
    const real fy = (real)(y & ((1 << ry) - 1)) * ((real)1 / (real)(1 << ry));  // exact: power of two
    if (D == 2) {
      s_off[gi][0] = g.offset + ky0 * nx;
      s_off[gi][R - 1] = g.offset + ky1 * nx;
      s_w[gi][0] = (real)1 - fy;
      s_w[gi][R - 1] = fy;
    } else {
      const int rz = n - g.l[D - 1];
      const int nz = 1 << g.l[D - 1];
      const int kz0 = z >> rz;
      const int kz1 = (kz0 + 1) & (nz - 1);
      const real fz = (real)(z & ((1 << rz) - 1)) * ((real)1 / (real)(1 << rz));
      s_off[gi][0] = g.offset + (kz0 * ny + ky0) * nx;
      s_off[gi][1 % R] = g.offset + (kz0 * ny + ky1) * nx;
      s_off[gi][2 % R] = g.offset + (kz1 * ny + ky0) * nx;
      s_off[gi][3 % R] = g.offset + (kz1 * ny + ky1) * nx;
      s_w[gi][0] = ((real)1 - fy) * ((real)1 - fz);
      s_w[gi][1 % R] = fy * ((real)1 - fz);
      s_w[gi][2 % R] = ((real)1 - fy) * fz;
      s_w[gi][3 % R] = fy * fz;
    }
    s_c[gi] = (real)g.coeff;
  }
  __syncthreads();

  // every (level, x index) of the levels Horner reads: each grid's term in
  // the run's precision (one rounding per product, like the component field
  // itself), then an error-free addition into the accumulator, so the
  // alternating-sign sum loses nothing to cancellation
  for (int e = threadIdx.x + (1 << lmin); e < 2 * N; e += blockDim.x) {
    const int l = 31 - __clz(e);
    const int kx = e - (1 << l);
    Acc<real> acc[D];
    for (int gi = s_start[l]; gi < s_start[l + 1]; ++gi) {
      const real c = s_c[gi];
#pragma unroll
      for (int m = 0; m < D; ++m) {
        const real* base = E + (size_t)m * S + kx;
        real val = s_w[gi][0] * base[s_off[gi][0]];
#pragma unroll
        for (int r = 1; r < R; ++r) val = fma(s_w[gi][r], base[s_off[gi][r]], val);
        acc[m].add(c * val);  // |c| is 1 or 2 (a power of two): exact
      }
    }
#pragma unroll
    for (int m = 0; m < D; ++m) A[m * 2 * N + e] = acc[m];
  }
  __syncthreads();
  for (int l = lmin; l < n; ++l) {
    const int cnt = 2 << l;  // size of level l+1
    const int half = 1 << l;
    for (int e2 = threadIdx.x; e2 < D * cnt; e2 += blockDim.x) {
      const int m = e2 >> (l + 1), e = e2 & (cnt - 1);
      Acc<real>* Am = A + m * 2 * N;
      const int k = e >> 1;
      Acc<real> v = Am[half + k];
      if (e & 1) {
        v.add_acc(Am[half + ((k + 1) & (half - 1))]);
        v.scale((real)0.5);
      }
      Am[cnt + e].add_acc(v);
    }
    __syncthreads();
  }
  // field energy: each thread sums the squares of its few nodes in the run's
  // precision; the block and the step reduce the partials in FP64
  real energy = (real)0;
  for (int e2 = threadIdx.x; e2 < D * N; e2 += blockDim.x) {
    const int m = e2 >> n, x = e2 & (N - 1);
    const Acc<real> v = A[m * 2 * N + N + x];
    const size_t o = (size_t)m * ND + (size_t)row * N + x;
    Ehi[o] = (real)v.hi();
    if (Elo) Elo[o] = (float)v.lo();
    energy = fma((real)v.hi(), (real)v.hi(), energy);
  }
  double tot = block_sum_double((double)energy, red);
  if (threadIdx.x == 0) partials[row] = tot;
  if (!fin.active) return;

  // The last block to finish reduces every row's partial (and the push's
  // kinetic-energy partials) in FP64, in a fixed order, so the step needs no
  // separate bookkeeping launch.
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(fin.counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double a = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) a += __ldcg(partials + i);
  const double fe = block_sum_double(a, red);
  double b = 0.0;
  if (fin.ke_partials)
    for (int i = threadIdx.x; i < fin.n_ke; i += blockDim.x) b += __ldcg(fin.ke_partials + i);
  const double ke = block_sum_double(b, red);
  if (threadIdx.x == 0) {
    DevDiag* dd = fin.dd;
    dd->field_energy_prev = dd->field_energy;
    dd->field_energy = fe * fin.fe_scale;
    if (fin.ke_partials) dd->kinetic_energy = ke;
    *fin.counter = 0u;
  }
}

template <typename real, int D>
int launch_combine(const GridDesc* grids, const LevelLists& ll, int lmin, const real* E, size_t S, int n, real* Ehi,
                   float* Elo, double* energy_partials, const CombineFinal& fin, cudaStream_t s) {
  const int N = 1 << n;
  unsigned rows = (unsigned)(D == 2 ? N : N * N);
  size_t smem = (size_t)D * 2 * N * sizeof(Acc<real>);
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_combine<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_combine<real, D><<<rows, 256, smem, s>>>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_COMB(real, D)                                                                                   \
  template int launch_combine<real, D>(const GridDesc*, const LevelLists&, int, const real*, size_t, int, real*, \
                                       float*, double*, const CombineFinal&, cudaStream_t);
SG_INST_COMB(float, 2)
SG_INST_COMB(float, 3)
SG_INST_COMB(double, 2)
SG_INST_COMB(double, 3)

}  // namespace sg
