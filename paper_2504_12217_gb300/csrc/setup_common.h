// Pieces of the GPU setup shared by the CRPC + PSQ key generator and the generic
// sparse-R1CS key generator (internal).
#pragma once
#include <vector>

#include "groth16.h"

namespace zkvc {

// Toxic waste in Montgomery form and derived constants of one setup.
struct SetupConsts {
  Fr tau, alpha, beta, gamma, delta, z;
  Fr tN1;   // tau^N - 1 = t(tau)
  Fr c;     // (tau^N - 1) / N
  Fr dinv, ginv;
  int bad;  // bit 0: non-canonical input, 1: tau^N = 1, 2: zero alpha..delta, 3: z in {0, 1}
};

// toxic: 6 canonical values (tau, alpha, beta, gamma, delta, z); dom_consts of the domain.
__global__ void k_setup_consts(const Fr* toxic, SetupConsts* sc, uint32_t logN, const Fr* dom_consts);

// L[k] = L_k(tau) for k < rows, one batched inversion per LAG_CHUNK rows and thread.
static constexpr int LAG_CHUNK = 32;
__global__ void k_lagrange(const SetupConsts* sc, const Fr* tw, size_t N, uint32_t rows, Fr* L);

__device__ __forceinline__ Fr pow_u32(Fr base, uint32_t e) {
  Fr r = Fr::one();
  while (e) {
    if (e & 1u) r = f_mul(r, base);
    base = f_sqr(base);
    e >>= 1;
  }
  return r;
}

__device__ __forceinline__ uint32_t bitrev_n(uint32_t x, uint32_t logN) { return __brev(x) >> (32 - logN); }

// Comb tables [d 2^(8 w)]G (w < 32, d < 256) of each group's generator, per device.
int fb_tables(G1A** t1, G2A** t2, cudaStream_t st);

// scalars (Montgomery) -> affine bases (Montgomery), in chunks of `chunk` through tmp.
template <class F>
int points_from_scalars(const Fr* scal, size_t n, const Affine<F>* T, Affine<F>* out, XYZZ<F>* tmp, size_t chunk,
                        cudaStream_t st);

// Canonical encodings of the points at the given indices (synchronises st).
template <class F>
int export_points(const Affine<F>* src, const std::vector<uint64_t>& idx, uint8_t* host_out, cudaStream_t st);

// RAII for temporaries of one setup call
struct DevTemps {
  std::vector<void*> ptrs;
  ~DevTemps() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  int alloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc(p, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("setup: cudaMalloc of %zu bytes: %s", count * sizeof(T), cudaGetErrorString(e));
      return ZKVC_ENOMEM;
    }
    ptrs.push_back(*p);
    return ZKVC_OK;
  }
};

}  // namespace zkvc
