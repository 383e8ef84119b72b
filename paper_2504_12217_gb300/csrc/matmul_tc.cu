// One-instance launcher of the tensor-core witness matmul (matmul_tc.cuh).
#include <algorithm>
#include <atomic>
#include <mutex>

#include "internal.h"
#include "matmul_tc.cuh"

namespace zkvc {

__global__ void __launch_bounds__(MM_THREADS) k_matmul_tc(const int8_t* __restrict__ X, const int8_t* __restrict__ W,
                                                          int32_t* __restrict__ Y, int a, int n, int b, int kslab,
                                                          int* flags, uint64_t first_wait_ns) {
  extern __shared__ __align__(128) uint8_t mm_dyn[];
  MatmulSmem& sm = *reinterpret_cast<MatmulSmem*>(mm_dyn);
  const int kb = blockIdx.z * kslab, ke = min(n, kb + kslab);
  matmul_tc_tile(X, W, Y, a, n, b, blockIdx.x * MM_M, blockIdx.y * MM_N, kb, ke, gridDim.z > 1, sm, flags,
                 first_wait_ns);
}

static std::once_flag g_mm_once;
static std::atomic<uint64_t> g_first_wait_ns{MATMUL_WAIT_NS};

void set_matmul_first_wait_ns(uint64_t ns) { g_first_wait_ns.store(ns, std::memory_order_relaxed); }

int matmul_init() {
  std::call_once(g_mm_once, [] {
    cudaFuncSetAttribute(k_matmul_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MatmulSmem));
  });
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

// K is split over CTAs (exact int32 atomics into a zeroed Y) while the output grid is
// smaller than the SM count, in slabs of whole 64-wide K tiles.
int matmul_i8(const int8_t* X, const int8_t* W, int32_t* Y, int a, int n, int b, int* flags, cudaStream_t st) {
  ZK_CHECK(a >= 1 && n >= 1 && b >= 1, ZKVC_EINVAL, "matmul: shape %d x %d x %d", a, n, b);
  ZK_CHECK((a + MM_N - 1) / MM_N <= 65535, ZKVC_EINVAL, "matmul: %d output rows exceed the grid", a);
  ZK_TRY(matmul_init());
  const int gm = (b + MM_M - 1) / MM_M, gn = (a + MM_N - 1) / MM_N;
  const int ktiles = (n + MM_BK - 1) / MM_BK;
  int splits = (device_sm_count() + gm * gn - 1) / (gm * gn);
  splits = std::max(1, std::min(splits, ktiles));
  const int per = (ktiles + splits - 1) / splits;
  splits = (ktiles + per - 1) / per;
  ZK_CHECK(splits <= 65535, ZKVC_EINVAL, "matmul: %d K slabs exceed the grid", splits);
  if (splits > 1) ZK_CUDA(cudaMemsetAsync(Y, 0, size_t(a) * b * sizeof(int32_t), st));
  dim3 grid((unsigned)gm, (unsigned)gn, (unsigned)splits);
  k_matmul_tc<<<grid, MM_THREADS, sizeof(MatmulSmem), st>>>(X, W, Y, a, n, b, per * MM_BK, flags,
                                                            g_first_wait_ns.load(std::memory_order_relaxed));
  ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

}  // namespace zkvc
