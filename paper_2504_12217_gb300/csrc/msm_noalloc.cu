// A variable-base G1 MSM that allocates nothing.
//
// Some callers cannot allocate device memory at all: code running inside a CUDA graph
// being captured, allocator-less embedded runtimes, or hosts whose device memory is
// fully reserved up front by another framework.  zkvc_msm_g1 needs a caller-provided
// workspace; this entry point instead keeps its scratch in one file-scope __device__
// array, resident on every GPU that loads the library until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it is only a
// host-side shadow), so the first call on each device -- with that device current --
// looks the real address up with cudaGetSymbolAddress and caches it.  That first call
// should therefore come before any stream capture.  Every call shares the one array: the
// MSM driver initialises all of its scratch it reads (bucket counters are cleared each
// call), so leftovers from a previous call are harmless, but two calls whose work
// overlaps on the GPU race on the array and must not be issued concurrently.
#include <map>
#include <mutex>

#include "msm.h"

#define ZKVC_MSM_NOALLOC_SCRATCH_BYTES (size_t(8) << 20)

namespace zkvc {

static __device__ __align__(256) uint8_t g_noalloc_scratch[ZKVC_MSM_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static std::map<int, void*> g_noalloc_addr;

// Device address of the scratch array on the current device (looked up once per device).
static int noalloc_scratch(void** out) {
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it == g_noalloc_addr.end()) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    ZK_CHECK(e == cudaSuccess && ptr != nullptr, ZKVC_ECUDA, "msm_g1_noalloc: cudaGetSymbolAddress failed: %s",
             cudaGetErrorString(e));
    it = g_noalloc_addr.emplace(dev, ptr).first;
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
