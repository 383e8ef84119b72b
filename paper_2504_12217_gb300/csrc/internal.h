// Internal declarations shared by the translation units of libzkvc (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "../../include/zkvc.h"

namespace zkvc {

void set_error(const char* fmt, ...);
const char* last_error_text();  // the calling thread's last error message

// Number of kernels this library has launched in the process (diagnostics).
void count_launch();
void count_launches(unsigned long long n);    // kernels of a replayed graph
void uncount_launches(unsigned long long n);  // kernels recorded into a graph, not run
unsigned long long launches_so_far();
#define ZK_COUNT_LAUNCH() ::zkvc::count_launch()

// Waits for the stream with a deadline (zkvc_set_wait_timeout_ms): ZKVC_OK when its work
// is done, ZKVC_ETIMEOUT when the deadline passes first (the work keeps running),
// ZKVC_ECUDA when the stream reports an error.
int wait_stream(cudaStream_t st, const char* what);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, cached
// per device); 1 when no device answers.  Launch shapes that aim at whole waves use it.
int device_sm_count();

// Y = X W (int8 x int8 -> int32, exact) on the tensor cores (matmul_tc.cu); sets bit 8
// of *flags if a tensor-core wait timed out.
int matmul_i8(const int8_t* X, const int8_t* W, int32_t* Y, int a, int n, int b, int* flags, cudaStream_t st);
// Limit of the matmul's first mbarrier waits for later launches (0: give up at once).
void set_matmul_first_wait_ns(uint64_t ns);

// Optional stage timers (CUDA events on the launching stream), enabled by
// zkvc_profile_enable; collected after the synchronising end of a prove call.
enum ProfStage : int {
  PS_WITNESS = 0,
  PS_NTT,
  PS_MSM_G1,
  PS_ACCUM_G1,   // the G1 bucket-accumulation kernel alone; units = bucket terms
  PS_MSM_G2,
  PS_ACCUM_G2,   // the G2 bucket-accumulation kernel alone; units = bucket terms
  PS_COMBINE,
  PS_MSM_SMALL,  // the small-digit G1 run and what follows it on its stream
  PS_COUNT
};
void prof_mark(int stage, bool begin, cudaStream_t st);

// NVTX range over the host-side enqueue of a prover stage ("zkvc/prove/ntt", ...), so that
// a profiler can select a stage's kernels by range (ncu --nvtx --nvtx-include); free when
// no tool is attached (NVTX is header-only and loads no library then).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
uint32_t* prof_units(int stage);  // pinned host slot for the stage's unit count, or null
void prof_collect();
bool prof_enabled();

#define ZK_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      ::zkvc::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return ZKVC_ECUDA;                                                                    \
    }                                                                                       \
  } while (0)

#define ZK_CHECK(cond, code, ...)       \
  do {                                  \
    if (!(cond)) {                      \
      ::zkvc::set_error(__VA_ARGS__);   \
      return (code);                    \
    }                                   \
  } while (0)

#define ZK_TRY(expr)             \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != ZKVC_OK) return rc_; \
  } while (0)

// Bump allocator over a caller-provided device workspace (256-byte aligned slices).
// bytes rounded up to a multiple of 256 (the alignment of every device buffer carved here)
inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

struct Arena {
  uint8_t* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  bool measuring = false;  // when true only sizes are accumulated
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    size_t at = off;
    off += bytes;
    if (measuring || base == nullptr) return nullptr;
    if (off > cap) return nullptr;
    return reinterpret_cast<T*>(base + at);
  }
  bool overflow() const { return !measuring && off > cap; }
};

inline uint32_t ceil_log2(size_t n) {
  uint32_t l = 0;
  while ((size_t(1) << l) < n) l++;
  return l;
}

}  // namespace zkvc
