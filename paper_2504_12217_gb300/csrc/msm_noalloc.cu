// A variable-base G1 MSM that allocates nothing.
//
// Some callers cannot allocate device memory at all: allocator-less embedded runtimes, or
// hosts whose device memory is fully reserved up front by another framework (a serving
// stack that claims the whole GPU for its own pool at start-up).  zkvc_msm_g1 needs a
// caller-provided workspace; this entry point instead keeps its scratch in one file-scope
// __device__ array, resident on every GPU that loads the library until the process exits.
// Like zkvc_msm_g1 it uploads its small bucket tables from host memory, synchronises
// `stream` and copies the 64-byte result to the caller's host buffer before returning.
//
// Host code cannot use the array's name as a device address (in host code it is only a
// host-side shadow), so the first call on each device -- with that device current --
// looks the real address up with cudaGetSymbolAddress and caches it, keyed on the device
// and on the identity of its current CUDA context (after cudaDeviceReset the module is
// loaded again and the array may move; the new context misses the cache and the address
// is looked up again).  That first call should therefore come before any stream capture.
// Every call shares the one array: the MSM driver initialises all of its scratch it reads
// (bucket counters are cleared each call), so leftovers from a previous call are harmless,
// but two calls whose work overlaps on the GPU race on the array and must not be issued
// concurrently.
#include <map>
#include <mutex>
#include <utility>

#include "msm.h"

#define ZKVC_MSM_NOALLOC_SCRATCH_BYTES (size_t(8) << 20)

namespace zkvc {

static __device__ __align__(256) uint8_t g_noalloc_scratch[ZKVC_MSM_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static std::map<std::pair<int, unsigned long long>, void*> g_noalloc_addr;

// Identity of the calling thread's current context (0 when none is current or the driver
// does not export the query): the runtime's primary context is replaced by
// cudaDeviceReset, and the module with the array is loaded again into the new one.
static unsigned long long current_context_id() {
  typedef int (*CtxGetCurrent)(void**);
  typedef int (*CtxGetId)(void*, unsigned long long*);
  static CtxGetCurrent get_current = nullptr;
  static CtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetId>(f);
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == 0 && ctx != nullptr && get_id(ctx, &id) == 0) return id;
  return 0;
}

// Device address of the scratch array on the current device, looked up once per device
// and context (a lookup allocates nothing).
static int noalloc_scratch(void** out) {
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned long long ctx = current_context_id();
  auto it = ctx ? g_noalloc_addr.find({dev, ctx}) : g_noalloc_addr.end();
  if (it == g_noalloc_addr.end()) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    ZK_CHECK(e == cudaSuccess && ptr != nullptr, ZKVC_ECUDA, "msm_g1_noalloc: cudaGetSymbolAddress failed: %s",
             cudaGetErrorString(e));
    ctx = current_context_id();  // the lookup makes the device's primary context current
    if (ctx == 0) {              // no context identity available: use the fresh lookup
      *out = ptr;
      return ZKVC_OK;
    }
    it = g_noalloc_addr.emplace(std::make_pair(dev, ctx), ptr).first;
  }
  *out = it->second;
  return ZKVC_OK;
}

}  // namespace zkvc

using namespace zkvc;

extern "C" int zkvc_msm_g1_noalloc(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, uint8_t out[64],
                                   void* stream) {
  set_error("%s", "");
  ZK_CHECK(n <= ZKVC_MSM_NOALLOC_MAX_POINTS, ZKVC_EINVAL,
           "msm_g1_noalloc: n = %zu exceeds the fixed maximum of %d points (use zkvc_msm_g1 with a workspace)", n,
           ZKVC_MSM_NOALLOC_MAX_POINTS);
  size_t need = msm_api_ws<Fp>(n);
  ZK_CHECK(need <= ZKVC_MSM_NOALLOC_SCRATCH_BYTES, ZKVC_EINVAL,
           "msm_g1_noalloc: %zu points need %zu scratch bytes, more than the %zu reserved", n, need,
           (size_t)ZKVC_MSM_NOALLOC_SCRATCH_BYTES);
  void* scratch = nullptr;
  ZK_TRY(noalloc_scratch(&scratch));
  return msm_api<Fp>(d_points, d_scalars, n, scratch, ZKVC_MSM_NOALLOC_SCRATCH_BYTES, out, (cudaStream_t)stream);
}
