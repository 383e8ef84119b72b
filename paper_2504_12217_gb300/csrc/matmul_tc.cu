// One-instance launcher of the tensor-core witness matmul (matmul_tc.cuh).
#include "internal.h"
#include "matmul_tc.cuh"

namespace zkvc {

__global__ void __launch_bounds__(MM_THREADS) k_matmul_tc(const int8_t* __restrict__ X, const int8_t* __restrict__ W,
                                                          int32_t* __restrict__ Y, int a, int n, int b, int* flags) {
  __shared__ MatmulSmem sm;
  matmul_tc_tile(X, W, Y, a, n, b, blockIdx.x * MM_M, blockIdx.y * MM_N, sm, flags);
}

int matmul_i8(const int8_t* X, const int8_t* W, int32_t* Y, int a, int n, int b, int* flags, cudaStream_t st) {
  ZK_CHECK(a >= 1 && n >= 1 && b >= 1, ZKVC_EINVAL, "matmul: shape %d x %d x %d", a, n, b);
  ZK_CHECK((b + MM_M - 1) / MM_M <= 0x7fffffff && (a + MM_N - 1) / MM_N <= 65535, ZKVC_EINVAL,
           "matmul: %d output rows exceed the grid", a);
  dim3 grid((unsigned)((b + MM_M - 1) / MM_M), (unsigned)((a + MM_N - 1) / MM_N));
  k_matmul_tc<<<grid, MM_THREADS, 0, st>>>(X, W, Y, a, n, b, flags); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

}  // namespace zkvc
