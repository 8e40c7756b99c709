// Cell-key sort without device allocation.
//
// sg_cell_sort obtains its scratch (key/index ping-pong buffers, digit
// histograms, scan totals, a status word) from the stream-ordered allocator
// on every call.  Some callers cannot do that: code that runs under a device
// memory budget owned by another allocator (a framework's caching allocator
// that holds all device memory), or latency-critical loops in which an
// allocation or a free may synchronise the device or fail under
// fragmentation.  For them, sg_cell_sort_static runs the same kernels on a
// fixed scratch area that is part of the library image: a file-scope device
// array of SG_CELL_SORT_STATIC_WORDS words, present on every GPU that loads
// the library for the life of the process.
//
// Host code cannot use the array's name as a device address (it denotes a
// host-side stand-in), so the first call on each device looks the address up
// with cudaGetSymbolAddress while that device is current and caches it.
// Every call shares the array and it keeps the previous call's contents:
// the only word that must start at zero (the status word) is cleared on the
// call's stream, everything else is fully rewritten before it is read.  Two
// calls whose work overlaps on the GPU (different streams, no ordering) race
// on the array.
#include <mutex>

#include "sg_kernels.cuh"

namespace sg {

// keys, index, key ping-pong (3 x max), digit histograms and scan totals of
// the radix sort, one status word, padding.
constexpr size_t kStaticMax = SG_CELL_SORT_STATIC_MAX;
constexpr size_t kStaticTiles = (kStaticMax + RS_TILE - 1) / RS_TILE;
constexpr size_t kStaticWords = 3 * kStaticMax + 256 * kStaticTiles + (256 * kStaticTiles) / 4096 + 1 + 64 + 16;
static_assert(kStaticWords <= SG_CELL_SORT_STATIC_WORDS, "scratch layout exceeds the declared size");

static __device__ __align__(256) uint32_t g_cell_sort_scratch[SG_CELL_SORT_STATIC_WORDS];

namespace {
std::mutex g_static_mu;
uint32_t* g_static_addr[256] = {};  // per device ordinal

int static_scratch(uint32_t** out) {
  int dev = 0;
  SG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("sg_cell_sort_static: device ordinal out of range");
    return SG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cell_sort_scratch);
    if (e != cudaSuccess) {
      set_error(std::string("sg_cell_sort_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return SG_ERR_CUDA;
    }
    g_static_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_static_addr[dev];
  return SG_OK;
}
}  // namespace

}  // namespace sg

using namespace sg;

extern "C" int sg_cell_sort_static(int precision, int dim, int level, size_t n, const void* const* u,
                                   uint32_t* keys_sorted, uint32_t* perm, uint32_t* counts, void* stream) {
  if (dim != 2 && dim != 3) {
    set_error("sg_cell_sort_static: dim must be 2 or 3");
    return SG_ERR_INVALID;
  }
  if (level < 1 || dim * level > 24) {
    set_error("sg_cell_sort_static: need 1 <= level and dim*level <= 24");
    return SG_ERR_INVALID;
  }
  if (precision != SG_FP32 && precision != SG_FP64) {
    set_error("sg_cell_sort_static: bad precision");
    return SG_ERR_INVALID;
  }
  if (n > kStaticMax) {
    set_error("sg_cell_sort_static: " + std::to_string(n) + " positions exceed the fixed scratch capacity of " +
              std::to_string(kStaticMax) + " (use sg_cell_sort)");
    return SG_ERR_SIZE;
  }
  if (n > 0 && (!u || !keys_sorted || !perm)) {
    set_error("sg_cell_sort_static: NULL pointer");
    return SG_ERR_INVALID;
  }
  for (int m = 0; n > 0 && m < dim; ++m)
    if (!u[m]) {
      set_error("sg_cell_sort_static: NULL position array");
      return SG_ERR_INVALID;
    }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cells = (size_t)1 << (dim * level);
  if (n == 0) {
    if (counts) SG_CUDA(cudaMemsetAsync(counts, 0, cells * 4, s));
    return SG_OK;
  }
  uint32_t* buf = nullptr;
  SG_TRY(static_scratch(&buf));
  uint32_t* keys = buf;
  uint32_t* vals = buf + kStaticMax;
  uint32_t* keys_alt = buf + 2 * kStaticMax;
  uint32_t* scr = buf + 3 * kStaticMax;
  const size_t scr_words = sort_scratch_words(n);
  if (3 * kStaticMax + scr_words + 1 > (size_t)SG_CELL_SORT_STATIC_WORDS) {
    set_error("sg_cell_sort_static: scan layout exceeds the fixed scratch capacity");
    return SG_ERR_SIZE;
  }
  unsigned* status = (unsigned*)(scr + scr_words);
  SG_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), s));  // the one word that must start at zero
  SortScratch sc;
  sort_scratch_bind(sc, scr, n);
  int st;
  if (precision == SG_FP32) {
    st = dim == 2 ? launch_keys_raw<float, 2>((const float* const*)u, n, level, keys, nullptr, nullptr, status, s)
                  : launch_keys_raw<float, 3>((const float* const*)u, n, level, keys, nullptr, nullptr, status, s);
  } else {
    st = dim == 2 ? launch_keys_raw<double, 2>((const double* const*)u, n, level, keys, nullptr, nullptr, status, s)
                  : launch_keys_raw<double, 3>((const double* const*)u, n, level, keys, nullptr, nullptr, status, s);
  }
  if (st != SG_OK) return st;
  bool in_alt = false;
  SG_TRY(radix_sort_pairs(keys, vals, keys_alt, perm, n, dim * level, true, sc, s, &in_alt));
  const uint32_t* ks = in_alt ? keys_alt : keys;
  const uint32_t* ps = in_alt ? perm : vals;
  SG_CUDA(cudaMemcpyAsync(keys_sorted, ks, n * 4, cudaMemcpyDeviceToDevice, s));
  if (ps != perm) SG_CUDA(cudaMemcpyAsync(perm, ps, n * 4, cudaMemcpyDeviceToDevice, s));
  if (counts) {
    SG_CUDA(cudaMemsetAsync(counts, 0, cells * 4, s));
    SG_TRY(launch_counts(keys_sorted, n, counts, s));
  }
  return SG_OK;
}
