// Signed combination of the component fields on the regular nodes:
//   E_comb(x_j) = sum_i c_i (P_i E_i)(x_j)
// (eq. sparse_filter's c_i and P_i of eq. restriction, applied to the
// fields).  Two kernels share the scheme below: a warp per line for lines of
// up to 1024 nodes (values in registers), a block per line beyond.  Block
// per line: one block per regular row (a y line in 2D, a (y, z) line in
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

// ---------------------------------------------------------------- warp-per-line combination
//
// For lines of at most 1024 nodes: one warp per (regular line, field
// component), the level-l partial sum held in registers (2^l / 32
// consecutive values per lane once 2^l >= 32, one value on 2^l lanes
// before).  Each Horner step prolongs in place (even nodes copy, odd nodes
// average the two neighbours, the right neighbour's first value by shuffle)
// and adds the transverse interpolation of the grids whose x level is the
// new level, read with vector loads.  No block barriers.
//
// FP32 path: the values are float pairs hi + lo carried without
// renormalisation: every hi addition is an error-free two_sum whose error
// goes to lo, so lo collects the exact rounding errors of hi and the pair
// stays accurate to ~2^-48 of the largest intermediate, whatever the
// cancellation; one final two_sum renormalises before the hi / lo planes
// are stored.  FP64 path: plain double.
template <typename real>
struct CAcc;
template <>
struct CAcc<float> {
  using term = float;  // type of one grid's interpolated, scaled term
  float hi, lo;
  static __device__ __forceinline__ CAcc zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ CAcc avg(const CAcc& a, const CAcc& b) {
    const ff s = two_sum(a.hi, b.hi);
    return {s.hi * 0.5f, (a.lo + b.lo + s.lo) * 0.5f};
  }
  static __device__ __forceinline__ CAcc add(const CAcc& a, const CAcc& b) {
    const ff s = two_sum(a.hi, b.hi);
    return {s.hi, a.lo + b.lo + s.lo};
  }
  static __device__ __forceinline__ CAcc first(float t) { return {t, 0.f}; }
  static __device__ __forceinline__ CAcc add_term(const CAcc& a, float t) {
    const ff s = two_sum(a.hi, t);
    return {s.hi, a.lo + s.lo};
  }
  __device__ __forceinline__ CAcc shfl(int src) const {
    return {__shfl_sync(0xffffffffu, hi, src), __shfl_sync(0xffffffffu, lo, src)};
  }
  __device__ __forceinline__ ff normalised() const { return two_sum(hi, lo); }
};
template <>
struct CAcc<double> {
  using term = double;
  double v;
  static __device__ __forceinline__ CAcc zero() { return {0.0}; }
  static __device__ __forceinline__ CAcc avg(const CAcc& a, const CAcc& b) { return {(a.v + b.v) * 0.5}; }
  static __device__ __forceinline__ CAcc add(const CAcc& a, const CAcc& b) { return {a.v + b.v}; }
  static __device__ __forceinline__ CAcc first(double t) { return {t}; }
  static __device__ __forceinline__ CAcc add_term(const CAcc& a, double t) { return {a.v + t}; }
  __device__ __forceinline__ CAcc shfl(int src) const { return {__shfl_sync(0xffffffffu, v, src)}; }
};

// FP32 fields combined with FP64 accumulation (sg_params.combine =
// SG_COMBINE_FP64): each grid's term c_i w E_i is formed in double, which
// is exact (c_i and the transverse weights w are dyadic, E_i a float), and
// the alternating-sign sum and the Horner prolongation run in double.  The
// result is split into hi + lo floats for the same output planes as the
// float-float accumulator.  GB300 issues double arithmetic at a small
// fraction of the float rate, so this variant is the slower one.
struct CAccD {
  using term = double;
  double v;
  static __device__ __forceinline__ CAccD zero() { return {0.0}; }
  static __device__ __forceinline__ CAccD avg(const CAccD& a, const CAccD& b) { return {(a.v + b.v) * 0.5}; }
  static __device__ __forceinline__ CAccD add(const CAccD& a, const CAccD& b) { return {a.v + b.v}; }
  static __device__ __forceinline__ CAccD first(double t) { return {t}; }
  static __device__ __forceinline__ CAccD add_term(const CAccD& a, double t) { return {a.v + t}; }
  __device__ __forceinline__ CAccD shfl(int src) const { return {__shfl_sync(0xffffffffu, v, src)}; }
  __device__ __forceinline__ ff normalised() const {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
  }
};

template <typename AC>
constexpr bool kFp64Acc = false;
template <>
constexpr bool kFp64Acc<CAccD> = true;

// Transverse interpolation weights and coarse-row offsets of one grid at
// regular line (y, z): the 2^(d-1) coarse x-lines that bracket the line,
// each weight times the grid's coefficient (dyadic products: exact).
template <typename real, int D>
struct RowTerm {
  int off[1 << (D - 1)];
  real w[1 << (D - 1)];
};

// The two level-lev nodes that bracket regular node y along one axis and
// the weight of the second: node-centred, y / 2^r in coarse units (r = n -
// lev); cell-centred, (y + 1/2) / 2^r - 1/2 = (2y + 1 - 2^r) / 2^(r+1), whose
// floor may be -1 (wrapped).  Both weights are dyadic: exact.
template <typename real, bool CELL>
__device__ __forceinline__ void bracket(int y, int n, int lev, int& k0, int& k1, real& f) {
  const int r = n - lev;
  const int nl = 1 << lev;
  if (!CELL) {
    k0 = y >> r;
    f = (real)(y & ((1 << r) - 1)) * ((real)1 / (real)(1 << r));
  } else {
    const int num = 2 * y + 1 - (1 << r);
    const int fl = num >> (r + 1);  // arithmetic shift: floor
    f = (real)(num - fl * (2 << r)) * ((real)1 / (real)(2 << r));
    k0 = fl & (nl - 1);
  }
  k1 = (k0 + 1) & (nl - 1);
}

template <typename real, int D, bool CELL>
__device__ __forceinline__ RowTerm<real, D> row_term(const GridDesc& g, int n, int y, int z) {
  RowTerm<real, D> t;
  const int nx = 1 << g.l[0];
  const int ny = 1 << g.l[1];
  int ky0, ky1;
  real fy;
  bracket<real, CELL>(y, n, g.l[1], ky0, ky1, fy);
  const real c = (real)g.coeff;
  if (D == 2) {
    t.off[0] = g.offset + ky0 * nx;
    t.off[(1 << (D - 1)) - 1] = g.offset + ky1 * nx;
    t.w[0] = c * ((real)1 - fy);
    t.w[(1 << (D - 1)) - 1] = c * fy;
  } else {
    int kz0, kz1;
    real fz;
    bracket<real, CELL>(z, n, g.l[D - 1], kz0, kz1, fz);
    constexpr int R = 1 << (D - 1);
    t.off[0] = g.offset + (kz0 * ny + ky0) * nx;
    t.off[1 % R] = g.offset + (kz0 * ny + ky1) * nx;
    t.off[2 % R] = g.offset + (kz1 * ny + ky0) * nx;
    t.off[3 % R] = g.offset + (kz1 * ny + ky1) * nx;
    t.w[0] = c * (((real)1 - fy) * ((real)1 - fz));
    t.w[1 % R] = c * (fy * ((real)1 - fz));
    t.w[2 % R] = c * (((real)1 - fy) * fz);
    t.w[3 % R] = c * (fy * fz);
  }
  return t;
}

// Adds, to the K consecutive values T[0..K) at x index x0.. (K and x0
// multiples of 4), c_i times the transverse interpolation of every grid of
// x level `level`; the grids' row terms come from this warp's shared-memory
// table.  Grid by grid, all of a grid's loads first (one latency per grid).
template <typename real, int D, int K, typename AC>
__device__ __forceinline__ void add_level_terms(AC* T, const RowTerm<real, D>* rt_tab, const int* lstart,
                                                int level, const real* __restrict__ Em, int x0) {
  using TT = typename AC::term;
  constexpr int R = 1 << (D - 1);
  for (int gi = lstart[level]; gi < lstart[level + 1]; ++gi) {
    const RowTerm<real, D> rt = rt_tab[gi];
    TT t[K];
#pragma unroll
    for (int k = 0; k < K; k += 4) {
      const V4<real> a = ld4(Em + rt.off[0] + x0 + k);
#pragma unroll
      for (int q = 0; q < 4; ++q) t[k + q] = (TT)rt.w[0] * (TT)a.x[q];
    }
#pragma unroll
    for (int r = 1; r < R; ++r) {
#pragma unroll
      for (int k = 0; k < K; k += 4) {
        const V4<real> a = ld4(Em + rt.off[r] + x0 + k);
#pragma unroll
        for (int q = 0; q < 4; ++q) t[k + q] = fma((TT)rt.w[r], (TT)a.x[q], t[k + q]);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) T[k] = AC::add_term(T[k], t[k]);
  }
}

// The same at one x index (lines with fewer than 4 values per lane).
template <typename real, int D, typename AC>
__device__ __forceinline__ AC level_term1(const RowTerm<real, D>* rt_tab, const int* lstart, int level,
                                          const real* __restrict__ Em, int x) {
  using TT = typename AC::term;
  constexpr int R = 1 << (D - 1);
  AC acc = AC::zero();
  bool first = true;
  for (int gi = lstart[level]; gi < lstart[level + 1]; ++gi) {
    const RowTerm<real, D> rt = rt_tab[gi];
    TT t = (TT)rt.w[0] * (TT)Em[rt.off[0] + x];
#pragma unroll
    for (int r = 1; r < R; ++r) t = fma((TT)rt.w[r], (TT)Em[rt.off[r] + x], t);
    acc = first ? AC::first(t) : AC::add_term(acc, t);
    first = false;
  }
  return acc;
}

// Cell-centred grids.  Linear interpolation through the centres of a
// level-l line is the node-centred interpolant of the level-(l+1) line
// whose odd nodes are the centres (g[2k+1] = E[k]) and whose even nodes are
// the midpoints (g[2k] = (E[k-1] + E[k]) / 2); the regular centres are the
// midpoints of the level-n nodes.  So the same Horner scheme runs with each
// grid entering one level higher as g, and the regular-centre values are
// (T[j] + T[j+1]) / 2 of its level-n result, plus the grids of x level n
// at their own centres.

// g of the grids of x level `level - 1` at Horner level `level`, index t.
template <typename real, int D, typename AC>
__device__ __forceinline__ AC cell_term1(const RowTerm<real, D>* rt_tab, const int* lstart, int level,
                                         const real* __restrict__ Em, int t) {
  if (level < 1) return AC::zero();
  const int lc = level - 1, nc = 1 << lc;
  if (t & 1) return level_term1<real, D, AC>(rt_tab, lstart, lc, Em, t >> 1);
  return AC::avg(level_term1<real, D, AC>(rt_tab, lstart, lc, Em, ((t >> 1) - 1) & (nc - 1)),
                 level_term1<real, D, AC>(rt_tab, lstart, lc, Em, t >> 1));
}

// Adds g of every grid of x level `level - 1` to the K >= 2 consecutive
// values T[0..K) at Horner-level index x0.. (x0 a multiple of K): the
// grid's K/2 centre values from x0/2 on (vector loads once K/2 >= 4) and
// the one before, periodically.
template <typename real, int D, int K, typename AC>
__device__ __forceinline__ void add_level_terms_cell(AC* T, const RowTerm<real, D>* rt_tab,
                                                     const int* lstart, int level, const real* __restrict__ Em,
                                                     int x0) {
  using TT = typename AC::term;
  constexpr int R = 1 << (D - 1);
  constexpr int H = K / 2;
  const int lc = level - 1, nc = 1 << lc;
  const int c0 = x0 >> 1, cm = (c0 - 1) & (nc - 1);
  for (int gi = lstart[lc]; gi < lstart[lc + 1]; ++gi) {
    const RowTerm<real, D> rt = rt_tab[gi];
    TT t[H + 1];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const real* row = Em + rt.off[r];
      const TT w = (TT)rt.w[r];
      const TT prev = (TT)row[cm];
      t[0] = r == 0 ? w * prev : fma(w, prev, t[0]);
      if constexpr (H >= 4) {
#pragma unroll
        for (int k = 0; k < H; k += 4) {
          const V4<real> a = ld4(row + c0 + k);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            t[1 + k + q] = r == 0 ? w * (TT)a.x[q] : fma(w, (TT)a.x[q], t[1 + k + q]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < H; ++k)
          t[1 + k] = r == 0 ? w * (TT)row[c0 + k] : fma(w, (TT)row[c0 + k], t[1 + k]);
      }
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      T[2 * j + 1] = AC::add_term(T[2 * j + 1], t[j + 1]);
      T[2 * j] = AC::add_term(T[2 * j], (TT)0.5 * (t[j] + t[j + 1]));
    }
  }
}

// One Horner step in the register phase: Vc values per lane -> 2 Vc, then
// add the new level's terms; recurse up to level n (2 Vc <= VMAX).
template <typename real, int D, int Vc, int VMAX, bool CELL, typename AC>
struct CombLevels {
  static __device__ __forceinline__ void run(AC* T, int& level, int n, int lane,
                                             const RowTerm<real, D>* rt_tab, const int* lstart,
                                             const real* __restrict__ Em) {
    if constexpr (2 * Vc <= VMAX) {
      const AC right = T[0].shfl((lane + 1) & 31);
#pragma unroll
      for (int i = Vc - 1; i >= 0; --i) {  // in place, high to low
        const AC nxt = (i == Vc - 1) ? right : T[i + 1];
        T[2 * i + 1] = AC::avg(T[i], nxt);
        T[2 * i] = T[i];
      }
      ++level;
      constexpr int K = 2 * Vc;
      if constexpr (CELL) {
        add_level_terms_cell<real, D, K, AC>(T, rt_tab, lstart, level, Em, lane * K);
      } else if constexpr (K >= 4) {
        add_level_terms<real, D, K, AC>(T, rt_tab, lstart, level, Em, lane * K);
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
          T[k] = AC::add(T[k], level_term1<real, D, AC>(rt_tab, lstart, level, Em, lane * K + k));
      }
      if (level < n) CombLevels<real, D, 2 * Vc, VMAX, CELL, AC>::run(T, level, n, lane, rt_tab, lstart, Em);
    }
  }
};

// Shared by both combination kernels: the last block to finish reduces the
// energy partials (and the push's kinetic-energy partials) in FP64, in a
// fixed order, so the step needs no separate bookkeeping launch.
__device__ __forceinline__ void combine_finalize(const double* partials, int n_part, const CombineFinal& fin,
                                                 double* red) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(fin.counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double a = 0.0;
  for (int i = threadIdx.x; i < n_part; i += blockDim.x) a += __ldcg(partials + i);
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

// Lines per block of the warp-per-line kernel (one warp per line and
// component) and the bytes of its row-term tables (one per line).
template <int D>
constexpr int combine_rows_per_block() { return 4; }  // 3D: 2 rows measured 16% slower
template <typename real, int D, int NC>
__host__ __device__ constexpr size_t combine_table_bytes(int ngl) {
  return ((size_t)combine_rows_per_block<D>() * ngl * sizeof(RowTerm<real, D>) + 15) / 16 * 16;
}
// Stride of the output between nodes: NC = D fields are stored
// node-interleaved (ec_stride), a single density plainly.
template <int D, int NC>
constexpr int combine_out_stride() { return NC == 1 ? 1 : ec_stride<D>(); }

template <typename real, int D, int V, int NC, bool CELL, typename AC>
__global__ void __launch_bounds__(32 * combine_rows_per_block<D>() * NC) k_combine_warp(const GridDesc* __restrict__ grids, LevelLists ll, int lmin,
                                                      const real* __restrict__ E, size_t S, int n,
                                                      real* __restrict__ Ehi, float* __restrict__ Elo,
                                                      double* __restrict__ partials, const CombineFinal fin) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int N = 1 << n;
  const int rows = D == 2 ? N : N * N;
  const size_t ND = (size_t)rows * N;
  const int wib = threadIdx.x >> 5;
  const int task = blockIdx.x * (blockDim.x >> 5) + wib;  // (row, component)
  const int lane = threadIdx.x & 31;
  const int m = task % NC, row = task / NC;
  const int y = row & (N - 1);
  const int z = D == 3 ? (row >> n) : 0;
  const real* Em = E + (size_t)m * S;
  __shared__ int s_start[18];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 18; ++i) s_start[i] = ll.start[i];  // constant indices: no local copy
  }
  const int ngl = ll.start[17];
  constexpr int RPB = combine_rows_per_block<D>();  // the block's lines: all NC components of each
  constexpr int DP = combine_out_stride<D, NC>();
  // one row-term table per line, shared by the line's NC component warps
  RowTerm<real, D>* rt_all = reinterpret_cast<RowTerm<real, D>*>(smem_raw);
  RowTerm<real, D>* rt_tab = rt_all + (size_t)(wib / NC) * ngl;
  // [RPB][N][DP] with one padding word after every V nodes (a lane's run), so
  // that the lanes' stores of one step fall in distinct banks
  real* stage = reinterpret_cast<real*>(smem_raw + combine_table_bytes<real, D, NC>(ngl));
  const int row0 = blockIdx.x * RPB;
  pdl_trigger();
  for (int e = threadIdx.x; e < RPB * ngl; e += blockDim.x) {
    const int r = e / ngl, gi = e - r * ngl;
    const int rr = row0 + r;  // the block's line r
    rt_all[e] = row_term<real, D, CELL>(grids[ll.grid[gi]], n, rr & (N - 1), D == 3 ? (rr >> n) : 0);
  }
  __syncthreads();
  pdl_wait();  // the solve's fields
  real energy = (real)0;
  double energy_d = 0.0;  // FP64 accumulation: the squares of the double results
  if (row < rows) {
    AC T[V];
    // coarse phase: one value on 2^level lanes, up to 32 values.  The terms
    // of every coarse level, pairs (l, x) with l in [level, ltop] and
    // x < 2^l, numbered p = 2^l - 2^level + x (at most 62), are computed
    // first, two pairs per lane (p = lane and lane + 32) so that every lane
    // works, and are handed to lane x of level l by shuffles.  Each term sums
    // its level's grids in the same order as before.  Cell-centred grids
    // enter one level higher.
    int level = min(CELL ? lmin + 1 : lmin, min(n, 5));
    const int ltop = min(n, 5);
    const int p0 = 1 << level;
    const int npairs = (2 << ltop) - p0;
    AC pv[2];
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      const int p = lane + 32 * sl;
      if (p < npairs) {
        const int l = 31 - __clz(p + p0);
        const int x = p + p0 - (1 << l);
        pv[sl] = CELL ? cell_term1<real, D, AC>(rt_tab, s_start, l, Em, x)
                      : level_term1<real, D, AC>(rt_tab, s_start, l, Em, x);
      } else {
        pv[sl] = AC::zero();
      }
    }
    // the level-l term of this lane's x (zero beyond 2^l); every lane shuffles
    auto coarse = [&](int l) {
      const int p = (1 << l) - p0 + lane;
      const AC a = pv[0].shfl(p & 31), b = pv[1].shfl(p & 31);
      return lane < (1 << l) ? ((p >> 5) ? b : a) : AC::zero();
    };
    T[0] = coarse(level);
#pragma unroll
    for (int j = 1; j < 6; ++j) {
      if (level < ltop) {
        const int h = 1 << level;
        const int k = lane >> 1;
        const AC a = T[0].shfl(k & (h - 1));
        const AC b = T[0].shfl((k + 1) & (h - 1));
        T[0] = (lane & 1) ? AC::avg(a, b) : a;
        ++level;
        const AC c = coarse(level);
        if (lane < (1 << level)) T[0] = AC::add(T[0], c);
      }
    }
    // register phase: 2^level / 32 consecutive values per lane
    if (level < n) CombLevels<real, D, 1, V, CELL, AC>::run(T, level, n, lane, rt_tab, s_start, Em);
    if constexpr (CELL) {  // to the regular centres, then the grids of x level n
      if (N >= 32) {
        const AC right = T[0].shfl((lane + 1) & 31);
#pragma unroll
        for (int k = 0; k < V; ++k) T[k] = AC::avg(T[k], k == V - 1 ? right : T[k + 1]);
        if constexpr (V >= 4) {
          add_level_terms<real, D, V, AC>(T, rt_tab, s_start, n, Em, lane * V);
        } else {
#pragma unroll
          for (int k = 0; k < V; ++k)
            T[k] = AC::add(T[k], level_term1<real, D, AC>(rt_tab, s_start, n, Em, lane * V + k));
        }
      } else {
        const AC right = T[0].shfl((lane + 1) & (N - 1));
        T[0] = AC::avg(T[0], right);
        if (lane < N) T[0] = AC::add(T[0], level_term1<real, D, AC>(rt_tab, s_start, n, Em, lane));
      }
    }
    // hi parts to the block's node-interleaved stage, lo planes straight out
    const size_t o0 = (size_t)m * ND + (size_t)row * N;
    const int nb = (row - row0) * N;  // first node of this line in the block
    real* srow = stage + (size_t)nb * DP + nb / V + m;  // node x at srow[x * DP + x / V]
    const int per = N >= 32 ? V : 1;
    if (N >= 32 || lane < N) {
      if constexpr (sizeof(real) == 4) {
        if constexpr (V >= 4) {
#pragma unroll
          for (int k = 0; k < V; k += 4) {
            ff v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              v[q] = T[k + q].normalised();
              if constexpr (kFp64Acc<AC>) energy_d = fma(T[k + q].v, T[k + q].v, energy_d);
              else energy = fmaf(v[q].hi, v[q].hi, energy);
              srow[(size_t)(lane * V + k + q) * DP + lane] = v[q].hi;
            }
            if (Elo)
              *reinterpret_cast<float4*>(Elo + o0 + (size_t)lane * V + k) =
                  make_float4(v[0].lo, v[1].lo, v[2].lo, v[3].lo);
          }
        } else {
#pragma unroll
          for (int k = 0; k < V; ++k)
            if (k < per) {
              const ff v = T[k].normalised();
              srow[(size_t)(lane * per + k) * DP + (lane * per + k) / V] = v.hi;
              if (Elo) Elo[o0 + (size_t)lane * per + k] = v.lo;
              if constexpr (kFp64Acc<AC>) energy_d = fma(T[k].v, T[k].v, energy_d);
              else energy = fmaf(v.hi, v.hi, energy);
            }
        }
      } else {
#pragma unroll
        for (int k = 0; k < V; ++k)
          if (k < per) {
            srow[(size_t)(lane * per + k) * DP + (lane * per + k) / V] = T[k].v;
            energy = fma(T[k].v, T[k].v, energy);
          }
      }
    }
  }
  __syncthreads();
  {  // the block's RPB lines are contiguous nodes: coalesced stores of the stage
    const int nreal = RPB * N * DP;
    real* dst = Ehi + (size_t)row0 * N * DP;
    for (int i = threadIdx.x; i < nreal; i += blockDim.x) dst[i] = stage[i + (i / DP) / V];
  }
  const double tot = warp_sum((double)energy + energy_d);
  if (lane == 0 && row < rows) partials[task] = tot;
  if (!fin.active) return;
  combine_finalize(partials, rows * NC, fin, red);
}

// ---------------------------------------------------------------- block-per-line combination (lines > 1024)

// Block-kernel accumulator of FP32 fields with FP64 accumulation (the
// counterpart of CAccD): double sum, split into hi + lo floats on output.
struct AccF64 {
  using term = double;
  double v = 0.0;
  __device__ __forceinline__ void add(double a) { v += a; }
  __device__ __forceinline__ void add_acc(const AccF64& o) { v += o.v; }
  __device__ __forceinline__ void scale(double s) { v *= s; }
  __device__ __forceinline__ float hi() const { return (float)v; }
  __device__ __forceinline__ float lo() const { return (float)(v - (double)(float)v); }
};
template <typename A>
constexpr bool kFp64BlockAcc = false;
template <>
constexpr bool kFp64BlockAcc<AccF64> = true;

template <typename real, int D, int NC, bool CELL, typename AccT>
__global__ void __launch_bounds__(256) k_combine(const GridDesc* __restrict__ grids, LevelLists ll, int lmin,
                                                 const real* __restrict__ E, size_t S, int n, real* __restrict__ Ehi,
                                                 float* __restrict__ Elo, double* __restrict__ partials,
                                                 const CombineFinal fin) {
  using TT = typename AccT::term;
  extern __shared__ unsigned char smem_raw[];
  AccT* A = reinterpret_cast<AccT*>(smem_raw);  // [NC][2N], level l of comp m at m*2N + [2^l, 2^(l+1))
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
    const int ny = 1 << g.l[1];
    int ky0, ky1;
    real fy;
    bracket<real, CELL>(y, n, g.l[1], ky0, ky1, fy);
    if (D == 2) {
      s_off[gi][0] = g.offset + ky0 * nx;
      s_off[gi][R - 1] = g.offset + ky1 * nx;
      s_w[gi][0] = (real)1 - fy;
      s_w[gi][R - 1] = fy;
    } else {
      int kz0, kz1;
      real fz;
      bracket<real, CELL>(z, n, g.l[D - 1], kz0, kz1, fz);
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

  // the transverse interpolation of grid gi, component m, at x index kx
  auto tval = [&](int gi, int m, int kx) {
    const real* base = E + (size_t)m * S + kx;
    TT val = (TT)s_w[gi][0] * (TT)base[s_off[gi][0]];
#pragma unroll
    for (int r = 1; r < R; ++r) val = fma((TT)s_w[gi][r], (TT)base[s_off[gi][r]], val);
    return val;
  };
  // every (level, x index) of the levels Horner reads: each grid's term in
  // the run's precision (one rounding per product, like the component field
  // itself), then an error-free addition into the accumulator, so the
  // alternating-sign sum loses nothing to cancellation.  Cell-centred grids
  // of x level l enter at level l+1 as centre values (odd) and midpoints
  // (even), as in the warp kernel.
  const int l0 = CELL ? min(lmin + 1, n) : lmin;
  for (int e = threadIdx.x + (1 << l0); e < 2 * N; e += blockDim.x) {
    const int l = 31 - __clz(e);
    const int kx = e - (1 << l);
    AccT acc[NC];
    const int lg = CELL ? l - 1 : l;
    for (int gi = s_start[lg]; gi < s_start[lg + 1]; ++gi) {
      const TT c = (TT)s_c[gi];
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        if (!CELL) {
          acc[m].add(c * tval(gi, m, kx));  // |c| is 1 or 2 (a power of two): exact
        } else if (kx & 1) {
          acc[m].add(c * tval(gi, m, kx >> 1));
        } else {
          const int nc = 1 << lg;
          acc[m].add((TT)0.5 * c * tval(gi, m, ((kx >> 1) - 1) & (nc - 1)));
          acc[m].add((TT)0.5 * c * tval(gi, m, kx >> 1));
        }
      }
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) A[m * 2 * N + e] = acc[m];
  }
  __syncthreads();
  for (int l = l0; l < n; ++l) {
    const int cnt = 2 << l;  // size of level l+1
    const int half = 1 << l;
    for (int e2 = threadIdx.x; e2 < NC * cnt; e2 += blockDim.x) {
      const int m = e2 >> (l + 1), e = e2 & (cnt - 1);
      AccT* Am = A + m * 2 * N;
      const int k = e >> 1;
      AccT v = Am[half + k];
      if (e & 1) {
        v.add_acc(Am[half + ((k + 1) & (half - 1))]);
        v.scale((TT)0.5);
      }
      Am[cnt + e].add_acc(v);
    }
    __syncthreads();
  }
  // field energy: each thread sums the squares of its few nodes in the run's
  // precision; the block and the step reduce the partials in FP64
  real energy = (real)0;
  double energy_d = 0.0;  // FP64 accumulation: the squares of the double results
  for (int e2 = threadIdx.x; e2 < NC * N; e2 += blockDim.x) {
    const int m = e2 >> n, x = e2 & (N - 1);
    AccT v = A[m * 2 * N + N + x];
    if (CELL) {  // to the regular centres, then the grids of x level n
      v.add_acc(A[m * 2 * N + N + ((x + 1) & (N - 1))]);
      v.scale((TT)0.5);
      for (int gi = s_start[n]; gi < s_start[n + 1]; ++gi) v.add((TT)s_c[gi] * tval(gi, m, x));
    }
    const size_t o = (size_t)m * ND + (size_t)row * N + x;
    Ehi[((size_t)row * N + x) * combine_out_stride<D, NC>() + m] = (real)v.hi();
    if (Elo) Elo[o] = (float)v.lo();
    if constexpr (kFp64BlockAcc<AccT>) energy_d = fma(v.v, v.v, energy_d);
    else energy = fma((real)v.hi(), (real)v.hi(), energy);
  }
  double tot = block_sum_double((double)energy + energy_d, red);
  if (threadIdx.x == 0) partials[row] = tot;
  if (!fin.active) return;
  combine_finalize(partials, (int)gridDim.x, fin, red);
}

template <typename real, int D, int V, int NC, bool CELL, typename AC>
static int launch_combine_warp(const GridDesc* grids, const LevelLists& ll, int lmin, const real* E, size_t S, int n,
                               real* Ehi, float* Elo, double* energy_partials, const CombineFinal& fin,
                               cudaStream_t s) {
  const int N = 1 << n;
  const long long rows = D == 2 ? N : (long long)N * N;
  constexpr int RPB = combine_rows_per_block<D>();
  const unsigned blocks = (unsigned)(rows / RPB);  // N >= 4: RPB divides the line count
  const size_t smem = combine_table_bytes<real, D, NC>(ll.start[17]) +
                      ((size_t)RPB * N * combine_out_stride<D, NC>() + (size_t)RPB * N / V) * sizeof(real);
  static bool attr_set = false;
  if (!attr_set && smem > 48 * 1024) {
    SG_CUDA(cudaFuncSetAttribute(k_combine_warp<real, D, V, NC, CELL, AC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    attr_set = true;
  }
  SG_CUDA(launch_pdl(k_combine_warp<real, D, V, NC, CELL, AC>, dim3(blocks), dim3(32 * RPB * NC), smem, s, grids, ll, lmin, E,
                     S, n, Ehi, Elo, energy_partials, fin));
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template <typename real, int D, int NC, bool CELL, typename AC, typename AccT>
static int launch_combine_nc(const GridDesc* grids, const LevelLists& ll, int lmin, const real* E, size_t S, int n,
                             real* Ehi, float* Elo, double* energy_partials, const CombineFinal& fin,
                             cudaStream_t s) {
  const int N = 1 << n;
  switch (N) {  // lines of up to 1024 nodes: warp per line, values in registers
    case 4:
    case 8:
    case 16:
    case 32:
      return launch_combine_warp<real, D, 1, NC, CELL, AC>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
    case 64:
      return launch_combine_warp<real, D, 2, NC, CELL, AC>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
    case 128:
      return launch_combine_warp<real, D, 4, NC, CELL, AC>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
    case 256:
      return launch_combine_warp<real, D, 8, NC, CELL, AC>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
    case 512:
      return launch_combine_warp<real, D, 16, NC, CELL, AC>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
    case 1024:
      return launch_combine_warp<real, D, 32, NC, CELL, AC>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
    default:
      break;
  }
  unsigned rows = (unsigned)(D == 2 ? N : N * N);
  size_t smem = (size_t)NC * 2 * N * sizeof(AccT);
  static bool attr_set = false;
  if (!attr_set) {
    SG_CUDA(cudaFuncSetAttribute(k_combine<real, D, NC, CELL, AccT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_combine<real, D, NC, CELL, AccT><<<rows, 256, smem, s>>>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin);
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template <typename real, int D, typename AC, typename AccT>
static int launch_combine_acc(const GridDesc* grids, const LevelLists& ll, int lmin, const real* E, size_t S, int n,
                              real* Ehi, float* Elo, double* energy_partials, const CombineFinal& fin, cudaStream_t s,
                              int ncomp, bool cell) {
  if (cell) {
    if (ncomp == 1)
      return launch_combine_nc<real, D, 1, true, AC, AccT>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
    return launch_combine_nc<real, D, D, true, AC, AccT>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
  }
  if (ncomp == 1)
    return launch_combine_nc<real, D, 1, false, AC, AccT>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
  return launch_combine_nc<real, D, D, false, AC, AccT>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s);
}

// fp64_acc selects FP64 accumulation of FP32 fields (CAccD / AccF64); the
// FP64 path always accumulates in double.
template <typename real, int D>
int launch_combine(const GridDesc* grids, const LevelLists& ll, int lmin, const real* E, size_t S, int n, real* Ehi,
                   float* Elo, double* energy_partials, const CombineFinal& fin, cudaStream_t s, int ncomp,
                   bool cell, bool fp64_acc) {
  if constexpr (sizeof(real) == 4) {
    if (fp64_acc)
      return launch_combine_acc<real, D, CAccD, AccF64>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin, s,
                                                        ncomp, cell);
  }
  return launch_combine_acc<real, D, CAcc<real>, Acc<real>>(grids, ll, lmin, E, S, n, Ehi, Elo, energy_partials, fin,
                                                            s, ncomp, cell);
}

#define SG_INST_COMB(real, D)                                                                                   \
  template int launch_combine<real, D>(const GridDesc*, const LevelLists&, int, const real*, size_t, int, real*, \
                                       float*, double*, const CombineFinal&, cudaStream_t, int, bool, bool);
SG_INST_COMB(float, 2)
SG_INST_COMB(float, 3)
SG_INST_COMB(double, 2)
SG_INST_COMB(double, 3)

}  // namespace sg
