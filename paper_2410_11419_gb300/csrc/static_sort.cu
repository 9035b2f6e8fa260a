// gs3_depth_order_static: the per-splat depth sort with its scratch memory in
// a file-scope device array instead of a caller workspace, for callers that
// may not allocate device memory.
#include <mutex>
#include <string>

#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr uint32_t kStaticMaxKeys = GS3_STATIC_SORT_MAX_KEYS;
constexpr int kStaticBlocks = (int)((kStaticMaxKeys + kSortTileItems - 1) / kSortTileItems);
constexpr size_t kStaticHistWords = 256ull * kStaticBlocks;
constexpr size_t kStaticScanWords = 256;  // >= scan_scratch_words(kStaticHistWords), padded
// ping-pong keys and values (3 of the 4 arrays; the caller's output is the 4th),
// radix histogram, scan partial sums
constexpr size_t kStaticWords = 3ull * kStaticMaxKeys + kStaticHistWords + kStaticScanWords;

static __device__ __align__(256) uint32_t g_static_scratch[kStaticWords];

// The array's device address per device, with the id of the CUDA context it
// was looked up in: a cudaDeviceReset destroys that context, and the module
// (with the array) may load at another address in the next one.
std::mutex g_mu;
uint32_t* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Id of the calling thread's current CUDA context (0 when it cannot be read),
// through the driver entry points cuCtxGetCurrent and cuCtxGetId.
unsigned long long current_context_id() {
  typedef int (*get_current_fn)(void**);
  typedef int (*get_id_fn)(void*, unsigned long long*);
  struct Fns {
    get_current_fn cur = nullptr;
    get_id_fn id = nullptr;
  };
  static const Fns fns = [] {
    Fns f;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.cur = reinterpret_cast<get_current_fn>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.id = reinterpret_cast<get_id_fn>(p);
    return f;
  }();
  if (!fns.cur || !fns.id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (fns.cur(&ctx) != 0 || !ctx || fns.id(ctx, &id) != 0) return 0;
  return id;
}

}  // namespace
}  // namespace gs3

using namespace gs3;

extern "C" gs3_status gs3_depth_order_static(const uint32_t* keys, uint32_t n, uint32_t* order_out,
                                             void* stream) {
  static_assert(kStaticScanWords >= (kStaticHistWords + kScanItems - 1) / kScanItems + 1,
                "scan scratch too small");
  if (n == 0) return GS3_OK;
  if (!keys || !order_out) {
    set_last_error("gs3_depth_order_static: null keys or order_out");
    return GS3_ERR_INVALID_ARG;
  }
  if (n > kStaticMaxKeys) {
    set_last_error("gs3_depth_order_static: n exceeds GS3_STATIC_SORT_MAX_KEYS (1048576)");
    return GS3_ERR_INVALID_ARG;
  }
  if (!device_range_ok(keys, (size_t)n * 4) || !device_range_ok(order_out, (size_t)n * 4)) {
    set_last_error("gs3_depth_order_static: keys or order_out is not device memory of n words");
    return GS3_ERR_INVALID_ARG;
  }
  int dev = 0;
  // cudaSetDevice makes the device's primary context current on this thread,
  // so that its id can be compared with the one the address was found in
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || cudaSetDevice(dev) != cudaSuccess) {
    set_last_error("gs3_depth_order_static: no usable current device");
    return GS3_ERR_CUDA;
  }
  uint32_t* base = nullptr;
  {
    // once per device and context, with that device current: the host-side
    // symbol is only a stand-in, the kernels need the array's device address
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        g_scratch_addr[dev] = nullptr;
        set_last_error("gs3_depth_order_static: cudaGetSymbolAddress of the scratch array failed");
        return GS3_ERR_CUDA;
      }
      g_scratch_addr[dev] = static_cast<uint32_t*>(p);
      g_scratch_ctx[dev] = current_context_id();
    }
    base = g_scratch_addr[dev];
  }
  uint32_t* k0 = base;
  uint32_t* v0 = base + kStaticMaxKeys;
  uint32_t* k1 = base + 2ull * kStaticMaxKeys;
  uint32_t* hist = base + 3ull * kStaticMaxKeys;
  uint32_t* scan = hist + kStaticHistWords;
  // four 8-bit passes over the 32-bit keys; the odd passes write the values
  // into the caller's output, so the last pass leaves the order there
  // an error left by an earlier, unrelated call on this thread is not this
  // call's: clear it so that the check below sees only these launches
  (void)cudaGetLastError();
  radix_sort_pairs(keys, nullptr, k0, v0, k1, order_out, n, 4, hist, scan,
                   reinterpret_cast<cudaStream_t>(stream));  // counts its own launches
  if (cudaGetLastError() != cudaSuccess) {
    set_last_error("gs3_depth_order_static: kernel launch failed");
    return GS3_ERR_CUDA;
  }
  return GS3_OK;
}
