// Shared device/host definitions of the sparse-grid PIC library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/sgpic.h"

#define SG_MAX_DIM 3
#define SG_THREADS 256

namespace sg {

// ---------------------------------------------------------------------------
// Error reporting (host).  Every CUDA runtime call goes through SG_CUDA; the
// first failure's text is kept per thread for sg_last_error().
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
const char* last_error();

struct Status {
  int code = SG_OK;
  explicit operator bool() const { return code != SG_OK; }
};

#define SG_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::sg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_) + " @ " + \
                      __FILE__ + ":" + std::to_string(__LINE__));                  \
      return SG_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

#define SG_TRY(...)             \
  do {                          \
    int s_ = (__VA_ARGS__);     \
    if (s_ != SG_OK) return s_; \
  } while (0)

// Kernel launches are counted (host side) so that callers can report how
// many library kernels ran; graph replays add the captured count.
void count_launch();
unsigned long long launches_so_far();
#define SG_CHECK_LAUNCH() \
  do {                    \
    ::sg::count_launch(); \
    SG_CUDA(cudaGetLastError()); \
  } while (0)

// Programmatic dependent launch (sm_90+).  A kernel launched with
// launch_pdl may start while its predecessor in the stream drains; it must
// call pdl_wait() before touching anything the predecessor writes (the wait
// returns once the predecessor has completed and its writes are visible).
// pdl_trigger() lets the successor start launching early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// device-side status bits (or-ed into a device word, read by diagnostics)
enum : unsigned {
  ST_NONFINITE = 1u,
  ST_KEY_RANGE = 2u,
  ST_BOUNDS = 4u,
};

// ---------------------------------------------------------------------------
// Particle arrays (structure of arrays) in the run's precision.
// ---------------------------------------------------------------------------
template <typename real, int D>
struct PArrays {
  real* u[D];  // fractional positions in [0,1)
  real* v[D];  // velocities
  real* w;     // charge per particle
  uint32_t* pid;  // original index
};

// Component-grid descriptor (device table).
struct GridDesc {
  int l[3];         // levels per axis (unused axes 0)
  int coeff;        // combination coefficient c_i
  int offset;       // offset of the grid in the component arenas (elements)
  int size;         // 2^|l|
  int run;          // owning run (batched serving); 0 for a single run
  int pad;
  double kfac[3];   // 2 pi / L_m (wavenumber of DFT index 1 along axis m)
  double vol;       // cell volume V_i = prod_m L_m / 2^l_m
};

// ---------------------------------------------------------------------------
// Morton (Z-order) key: bit b of axis m -> key bit b*D + m.
// ---------------------------------------------------------------------------
// Spread the low bits of x so that bit b lands on bit 2b (resp. 3b): the
// usual mask-and-shift interleave, valid for x < 2^16 (resp. 2^10).
__host__ __device__ __forceinline__ uint32_t spread2(uint32_t x) {
  x &= 0x0000FFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t x) {
  x &= 0x000003FFu;
  x = (x | (x << 16)) & 0xFF0000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

template <int D>
__host__ __device__ __forceinline__ uint32_t morton_key(const int* c, int /*n*/) {
  if (D == 2) return spread2((uint32_t)c[0]) | (spread2((uint32_t)c[1]) << 1);
  return spread3((uint32_t)c[0]) | (spread3((uint32_t)c[1]) << 1) | (spread3((uint32_t)c[D - 1]) << 2);
}

// Cell index floor(u 2^n) of a position already wrapped into [0,1).  The
// scaling by a power of two is exact, so the truncation equals the floor of
// the exact product in either precision.
template <typename real>
__device__ __forceinline__ int cell_of(real u, int n, int N) {
  int c = (int)(u * (real)N);
  return c < 0 ? 0 : (c >= N ? N - 1 : c);
}

// u - floor(u), with a rounded-up 1 mapped to 0 (periodic wrap into [0,1)).
__device__ __forceinline__ float sg_floor(float x) { return floorf(x); }
__device__ __forceinline__ double sg_floor(double x) { return ::floor(x); }

template <typename real>
__device__ __forceinline__ real wrap_unit(real u) {
  real w = u - sg_floor(u);
  return w >= (real)1 ? (real)0 : w;
}

// ---------------------------------------------------------------------------
// Float-float ("double-float") arithmetic: an unevaluated sum hi + lo of two
// floats carrying ~48 significant bits, used for the signed combination and
// the energy sums of the FP32 path.  Error-free transformations after Knuth
// (TwoSum) and the fused-multiply-add product (TwoProd).
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return two_sum(s.hi, lo);  // renormalise
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  return two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ ff ff_scale(ff a, float s) {  // s a power of two: exact
  return {a.hi * s, a.lo * s};
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Accumulator selection: float-float for the FP32 path, plain double for the
// FP64 path.
template <typename real>
struct Acc;

template <>
struct Acc<float> {
  using term = float;
  ff v{0.f, 0.f};
  __device__ __forceinline__ void add_prod(float a, float b) { v = ff_add(v, two_prod(a, b)); }
  __device__ __forceinline__ void add(float a) { v = ff_add_f(v, a); }
  __device__ __forceinline__ void add_acc(const Acc<float>& o) { v = ff_add(v, o.v); }
  __device__ __forceinline__ void scale(float s) { v = ff_scale(v, s); }
  __device__ __forceinline__ double to_double() const { return ff_to_double(v); }
  __device__ __forceinline__ float hi() const { return v.hi; }
  __device__ __forceinline__ float lo() const { return v.lo; }
};

template <>
struct Acc<double> {
  using term = double;
  double v = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void add(double a) { v += a; }
  __device__ __forceinline__ void add_acc(const Acc<double>& o) { v += o.v; }
  __device__ __forceinline__ void scale(double s) { v *= s; }
  __device__ __forceinline__ double to_double() const { return v; }
  __device__ __forceinline__ double hi() const { return v; }
  __device__ __forceinline__ double lo() const { return 0.0; }
};

// Four consecutive values with 16-byte vector loads / stores (the arrays
// come from cudaMalloc and every vector index is a multiple of 4).
template <typename real>
struct V4 {
  real x[4];
};

__device__ __forceinline__ V4<float> ld4(const float* p) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  return {{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.x[0], v.x[1], v.x[2], v.x[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.x[0], v.x[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.x[2], v.x[3]);
}

// Complex value in the run's precision.
template <typename real>
struct cplx {
  real x, y;
};

// ---------------------------------------------------------------------------
// Block-wide reductions.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ff w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, w);
  }
  return v;
}

// Sum one double per thread over the block; result valid in thread 0.
__device__ __forceinline__ double block_sum_double(double v, double* sh /* >= 32 */) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

}  // namespace sg
