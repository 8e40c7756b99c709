// Gather + push (Section 2, steps 3-4): CIC interpolation of the combined
// field (same shape as the deposit) plus the linear external field, then a
// leapfrog kick (Boris rotation when B != 0) and the drift
// x^{n+1} = x^n + v^{n+1/2} dt, wrapped into the periodic box.  Each thread
// also adds 0.5 m_p v^{n-1/2}.v^{n+1/2} to the time-centred kinetic energy.
//
// Each thread advances four consecutive particles per iteration with 16-byte
// vector loads and stores.  On a sort step the kernel also emits the tile key
// of every new position (the counting sort's keys; k_tile_hist counts them)
// and adds sum (cell key + 1) to the checksum.
#include "sg_kernels.cuh"

namespace sg {

static __device__ __forceinline__ bool finite_r(float x) { return isfinite(x); }
static __device__ __forceinline__ bool finite_r(double x) { return isfinite(x); }


// Kinetic-energy accumulator of one thread: FP32 path a float pair whose
// low part collects the exact rounding error of every addition (two_sum);
// FP64 path plain double.  Partials are reduced in FP64.
template <typename real>
struct KeAcc;
template <>
struct KeAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const ff s = two_sum(hi, x);
    hi = s.hi;
    lo += s.lo;
  }
  __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
};
template <>
struct KeAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double to_double() const { return v; }
};

// Node left of the gather position s = u * 2^n - shift in [-1/2, 2^n)
// (shift 1/2 on cell-centred grids), wrapped, and the offset from it.  FP32:
// floor through the 1.5 * 2^23 rounding trick (no conversion instruction);
// a position exactly on a node of odd index may land in the cell below
// with offset 1, which interpolates the same node value with weight 1.
// FP64: floor.
__device__ __forceinline__ void gather_cell(float s, int mask, int& c, float& f) {
  const float t = (s - 0.5f) + 12582912.0f;
  c = (__float_as_int(t) - 0x4B400000) & mask;
  f = s - (t - 12582912.0f);
}
__device__ __forceinline__ void gather_cell(double s, int mask, int& c, double& f) {
  const double fl = floor(s);
  c = (int)fl & mask;
  f = s - fl;
}

// Periodic wrap of a drifted position: u - floor(u), a rounded-up 1 mapped
// to 0.  A drift of less than one box per step needs only a compare and an
// add of +-1 (the same operation floor would select); larger ones take floor.
template <typename real>
__device__ __forceinline__ real wrap_drifted(real u) {
  real w = u < (real)0 ? u + (real)1 : (u >= (real)1 ? u - (real)1 : u);
  if (w < (real)0 || w >= (real)1) w = u - sg_floor(u);
  return w >= (real)1 ? (real)0 : w;
}

// The combined field at one node: one vector load from the node-interleaved
// array.
template <typename real, int D>
__device__ __forceinline__ void load_node_field(const real* __restrict__ Ec, unsigned node, real (&e)[D]) {
  if constexpr (sizeof(real) == 4 && D == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(Ec) + node);
    e[0] = t.x;
    e[D - 1] = t.y;
  } else if constexpr (sizeof(real) == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(Ec) + node);
    e[0] = t.x;
    e[1 % D] = t.y;
    e[D - 1] = t.z;
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2*>(Ec) + (size_t)node * (ec_stride<D>() / 2));
    e[0] = (real)a.x;
    e[1 % D] = (real)a.y;
    if constexpr (D == 3) e[D - 1] = (real)__ldg(Ec + (size_t)node * ec_stride<D>() + 2);
  }
}

// Advance one particle in registers.
template <typename real, int D>
__device__ __forceinline__ void push_one(real (&u)[D], real (&v)[D], real w, int n, const real* __restrict__ Ec,
                                         size_t ND, const PushParams<real>& pp, KeAcc<real>& ke, bool& bad) {
  const int N = 1 << n;
  const int mask = N - 1;
  const real half = (real)0.5;
  int c[D];
  real f[D], E[D];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    gather_cell(u[m] * (real)N - pp.shift, mask, c[m], f[m]);
    E[m] = (real)0;
  }
#pragma unroll
  for (int corner = 0; corner < (1 << D); ++corner) {
    real wgt = (real)1;
    unsigned node = 0, gs = 1;  // 2^{dn} <= 2^24 nodes
#pragma unroll
    for (int m = 0; m < D; ++m) {
      int b = (corner >> m) & 1;
      wgt *= b ? f[m] : ((real)1 - f[m]);
      node += (unsigned)((c[m] + b) & mask) * gs;
      gs *= (unsigned)N;
    }
    real e[D];
    load_node_field<real, D>(Ec, node, e);
#pragma unroll
    for (int m = 0; m < D; ++m) E[m] += wgt * e[m];
  }
  if (pp.has_eext) {
#pragma unroll
    for (int m = 0; m < D; ++m) E[m] += pp.eext[m] * (u[m] - half);
  }
  real vm[D];
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
      const real a0 = vm[0], a1 = vm[1], a2 = vm[D - 1];
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
    real vn = vm[m] + hk * E[m];
    dot += v[m] * vn;
    bad |= !finite_r(vn);
    v[m] = vn;
  }
  ke.add(w * pp.ke_fac * dot);
  if (pp.drift) {
#pragma unroll
    for (int m = 0; m < D; ++m) {
      real un = wrap_drifted(u[m] + v[m] * pp.dt_over_L[m]);
      bad |= !finite_r(un);
      u[m] = un;
    }
  }
}

// Tile key (Morton key of the level-(n - shift) cell) of a wrapped position;
// also returns the level-n key for the checksum.
template <typename real, int D>
__device__ __forceinline__ uint32_t tile_key(const real (&u)[D], int n, int shift, uint32_t* full) {
  const int N = 1 << n;
  int c[D];
#pragma unroll
  for (int m = 0; m < D; ++m) c[m] = cell_of(u[m], n, N);
  uint32_t k = morton_key<D>(c, n);
  *full = k;
  return k >> (D * shift);
}

template <typename real, int D>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? (D == 2 ? 4 : 2) : 0) k_push(PArrays<real, D> p, size_t np, int n, const real* __restrict__ Ec,
                                              PushParams<real> pp, double* __restrict__ ke_partials,
                                              unsigned* status, SortFuse sf) {
  __shared__ double red[32];
  const int N = 1 << n;
  const size_t ND = (size_t)N * (D == 2 ? N : (size_t)N * N);
  pdl_wait();  // the combined field (no-op when launched without the attribute)
  KeAcc<real> ke;
  bool bad = false;
  unsigned long long cks = 0;
  const size_t nvec = np >> 2;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t iv = (size_t)blockIdx.x * blockDim.x + threadIdx.x; iv < nvec; iv += stride) {
    const size_t i0 = iv << 2;
    V4<real> U[D], Vv[D];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      U[m] = ld4(p.u[m] + i0);
      Vv[m] = ld4(p.v[m] + i0);
    }
    const V4<real> W = ld4(p.w + i0);
    uint32_t tiles[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      real u[D], v[D];
#pragma unroll
      for (int m = 0; m < D; ++m) {
        u[m] = U[m].x[j];
        v[m] = Vv[m].x[j];
      }
      push_one<real, D>(u, v, W.x[j], n, Ec, ND, pp, ke, bad);
#pragma unroll
      for (int m = 0; m < D; ++m) {
        U[m].x[j] = u[m];
        Vv[m].x[j] = v[m];
      }
      if (sf.keys) {
        uint32_t full;
        tiles[j] = tile_key<real, D>(u, n, sf.tile_shift, &full);
        cks += (unsigned long long)full + 1ull;
      }
    }
#pragma unroll
    for (int m = 0; m < D; ++m) {
      if (pp.drift) st4(p.u[m] + i0, U[m]);
      st4(p.v[m] + i0, Vv[m]);
    }
    if (sf.keys) *reinterpret_cast<uint4*>(sf.keys + i0) = make_uint4(tiles[0], tiles[1], tiles[2], tiles[3]);
  }
  // ragged tail (np not a multiple of 4): block 0 takes it particle by particle
  if (blockIdx.x == 0) {
    const size_t i = (nvec << 2) + threadIdx.x;
    const bool valid = i < np;
    if (valid) {
      real u[D], v[D];
#pragma unroll
      for (int m = 0; m < D; ++m) {
        u[m] = p.u[m][i];
        v[m] = p.v[m][i];
      }
      push_one<real, D>(u, v, p.w[i], n, Ec, ND, pp, ke, bad);
#pragma unroll
      for (int m = 0; m < D; ++m) {
        if (pp.drift) p.u[m][i] = u[m];
        p.v[m][i] = v[m];
      }
      if (sf.keys) {
        uint32_t full;
        uint32_t t = tile_key<real, D>(u, n, sf.tile_shift, &full);
        sf.keys[i] = t;
        cks += (unsigned long long)full + 1ull;
      }
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
  if (sf.checksum) {
    cks = warp_sum(cks);
    if ((threadIdx.x & 31) == 0 && cks) atomicAdd(sf.checksum, cks);
  }
  double tot = block_sum_double(ke.to_double(), red);
  if (threadIdx.x == 0 && ke_partials) ke_partials[blockIdx.x] = tot;
}

// Blocks of the push: one resident wave (SMs x blocks per SM at the kernel's
// register budget), each block walking its particles grid-stride; fewer for
// small runs.  A second wave of blocks measured 7% slower on the 2D step.
template <typename real, int D>
int push_blocks(size_t np) {
  static int cap = 0;
  if (!cap) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<real, D>, 256, 0) == cudaSuccess &&
        sms > 0 && per_sm > 0) {
      cap = sms * per_sm;
    } else {
      cudaGetLastError();
      cap = 152 * 4;
    }
  }
  size_t b = (np / 4 + 255) / 256;
  if (b > (size_t)cap) b = (size_t)cap;
  if (b == 0) b = 1;
  return (int)b;
}

template <typename real, int D>
int launch_push(const PArrays<real, D>& p, size_t np, int n, const real* Ecomb, PushParams<real> pp,
                double* ke_partials, unsigned* status, const SortFuse& sf, cudaStream_t s, int blocks) {
  if (blocks <= 0) blocks = push_blocks<real, D>(np);
  if (sf.keys)  // sort steps: memsets precede the push
    k_push<real, D><<<blocks, 256, 0, s>>>(p, np, n, Ecomb, pp, ke_partials, status, sf);
  else
    SG_CUDA(launch_pdl(k_push<real, D>, dim3(blocks), dim3(256), 0, s, p, np, n, Ecomb, pp, ke_partials, status, sf));
  SG_CHECK_LAUNCH();
  return SG_OK;
}

#define SG_INST_PUSH(real, D)                                                                           \
  template int launch_push<real, D>(const PArrays<real, D>&, size_t, int, const real*, PushParams<real>, \
                                    double*, unsigned*, const SortFuse&, cudaStream_t, int);             \
  template int push_blocks<real, D>(size_t);
SG_INST_PUSH(float, 2)
SG_INST_PUSH(float, 3)
SG_INST_PUSH(double, 2)
SG_INST_PUSH(double, 3)

}  // namespace sg
