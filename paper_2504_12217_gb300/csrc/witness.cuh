// Device bodies of the witness, CRPC and proof-encoding steps, shared by the one-proof
// prover and the batched prover (each kernel there maps its blocks to these bodies).
//
// CRPC (zkVC Sec. III-A): with z drawn at setup, the matmul Y = X W is proven through
// the n row constraints a_k b_k = c_k, where a_k = sum_i z^(ib) x_ik and
// b_k = sum_j z^j w_kj, and Y(z) = sum_(i,j) z^(ib + j) y_ij.  PSQ (Sec. III-B) chains
// the products through prefix sums S_k = S_(k-1) + c_k, closing S_(n-2) + c_(n-1) = Y(z).
#pragma once
#include "curve.cuh"

namespace zkvc {

// Sum over the block of per-thread Fr values (blockDim.x = 256, sh of 256 entries).
__device__ __forceinline__ Fr block_sum(Fr v, Fr* sh) {
  st_field(sh + threadIdx.x, v);
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) st_field(sh + threadIdx.x, f_add(ld_field(sh + threadIdx.x), ld_field(sh + threadIdx.x + s)));
    __syncthreads();
  }
  Fr r = ld_field(sh);
  __syncthreads();
  return r;
}

// Block body for row k < n: a_k and b_k (256 threads).
__device__ __forceinline__ void crpc_ab_row(const int8_t* __restrict__ X, const int8_t* __restrict__ W,
                                            const Fr* __restrict__ zA, const Fr* __restrict__ zB, int a, int n, int b,
                                            int k, Fr* ak, Fr* bk, Fr* sh) {
  Fr s = Fr::zero();
  for (int i = threadIdx.x; i < a; i += blockDim.x)
    s = f_add(s, f_mul(ld_field(zA + i), f_from_int<FrCfg>(X[size_t(i) * n + k])));
  Fr av = block_sum(s, sh);
  s = Fr::zero();
  for (int j = threadIdx.x; j < b; j += blockDim.x)
    s = f_add(s, f_mul(ld_field(zB + j), f_from_int<FrCfg>(W[size_t(k) * b + j])));
  Fr bv = block_sum(s, sh);
  if (threadIdx.x == 0) {
    st_field(ak + k, av);
    st_field(bk + k, bv);
  }
}

// Block body for row i < a of Y: z^(ib) sum_j z^j y_ij (256 threads).
__device__ __forceinline__ void crpc_y_row(const int32_t* __restrict__ Y, const Fr* __restrict__ zA,
                                           const Fr* __restrict__ zB, int b, int i, Fr* part, Fr* sh) {
  Fr s = Fr::zero();
  for (int j = threadIdx.x; j < b; j += blockDim.x)
    s = f_add(s, f_mul(ld_field(zB + j), f_from_int<FrCfg>(Y[size_t(i) * b + j])));
  Fr v = block_sum(s, sh);
  if (threadIdx.x == 0) st_field(part + i, f_mul(v, ld_field(zA + i)));
}

// Block body (1024 threads, sh of 1024 entries): c_k = a_k b_k, the prefix sums
// S_k = c_0 + ... + c_k for k <= n - 2, the closing check against Y(z) (flag bit 1), and
// the first n domain evaluations A_ev = a, B_ev = b, C_ev = c.
// Fr value of lane src (shuffle of the eight words); every lane of the warp calls it
__device__ __forceinline__ Fr fr_shfl_up(const Fr& x, int d) {
  Fr r;
#pragma unroll
  for (int i = 0; i < 8; i++) r.v[i] = __shfl_up_sync(0xffffffffu, x.v[i], d);
  return r;
}
__device__ __forceinline__ Fr fr_shfl_down(const Fr& x, int d) {
  Fr r;
#pragma unroll
  for (int i = 0; i < 8; i++) r.v[i] = __shfl_down_sync(0xffffffffu, x.v[i], d);
  return r;
}

// Inclusive scan of Fr sums over a warp (five shuffle rounds); every lane calls it.
__device__ __forceinline__ Fr warp_scan_fr(Fr v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const Fr u = fr_shfl_up(v, d);
    if (lane >= d) v = f_add(v, u);
  }
  return v;
}

__device__ __forceinline__ void psq_chain(const Fr* __restrict__ ak, const Fr* __restrict__ bk,
                                          const Fr* __restrict__ ypart, int a, int n, Fr* S, Fr* Aev, Fr* Bev, Fr* Cev,
                                          int* flags, Fr* sh) {
  const int T = blockDim.x;
  const int per = (n + T - 1) / T;
  const int k0 = threadIdx.x * per;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Fr local = Fr::zero();
  for (int k = k0; k < k0 + per && k < n; k++) {
    Fr a_ = ld_field(ak + k), b_ = ld_field(bk + k);
    Fr c = f_mul(a_, b_);
    st_field(Aev + k, a_);
    st_field(Bev + k, b_);
    st_field(Cev + k, c);
    local = f_add(local, c);
  }
  // inclusive scan of the per-thread sums: within each warp by shuffles, then over the
  // warps' totals by warp 0
  const Fr incl = warp_scan_fr(local);
  if (lane == 31) st_field(sh + wid, incl);
  __syncthreads();
  if (wid == 0) {
    Fr t = lane < T / 32 ? ld_field(sh + lane) : Fr::zero();
    t = warp_scan_fr(t);
    st_field(sh + 32 + lane, t);  // inclusive totals of warps 0 .. lane
  }
  __syncthreads();
  Fr run = f_sub(incl, local);  // this thread's exclusive prefix within its warp
  if (wid) run = f_add(run, ld_field(sh + 32 + wid - 1));
  for (int k = k0; k < k0 + per && k < n; k++) {
    run = f_add(run, ld_field(Cev + k));  // c_k as this thread stored it above
    if (k < n - 1) st_field(S + k, run);
  }
  // closing check against Y(z) = sum_i ypart_i (warp 1: strided sums, then a shuffle tree)
  if (wid == (T > 32 ? 1 : 0)) {
    Fr yz = Fr::zero();
    for (int i = lane; i < a; i += 32) yz = f_add(yz, ld_field(ypart + i));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) yz = f_add(yz, fr_shfl_down(yz, d));
    if (lane == 0) {
      const Fr total = ld_field(sh + 32 + (T / 32) - 1);  // S_(n-2) + c_(n-1)
      if (total != yz) atomicOr(flags, 1);
    }
  }
}

// Domain row k >= n: A_ev[n + v] = w_v for v = 0 .. l (one, X, Y), zeros elsewhere
// (the input-consistency rows).
__device__ __forceinline__ void domain_rest_row(const int8_t* __restrict__ X, const int32_t* __restrict__ Y, int n,
                                                uint32_t an, uint32_t l, size_t k, Fr* Aev, Fr* Bev, Fr* Cev) {
  size_t v = k - n;
  Fr w = Fr::zero();
  if (v == 0)
    w = Fr::one();
  else if (v <= an)
    w = f_from_int<FrCfg>(X[v - 1]);
  else if (v <= l)
    w = f_from_int<FrCfg>(Y[v - 1 - an]);
  st_field(Aev + k, w);
  st_field(Bev + k, Fr::zero());
  st_field(Cev + k, Fr::zero());
}

__device__ __forceinline__ bool canonical_fr(const Fr& x) {
  for (int i = 7; i >= 0; i--) {
    uint32_t m = mod_limb<FrCfg>(i);
    if (x.v[i] != m) return x.v[i] < m;
  }
  return false;
}

__device__ __forceinline__ void write_canon(uint8_t* out, const Fp& x) {
  Fp c = f_from_mont(x);
  for (int i = 0; i < 8; i++) {
    out[4 * i] = (uint8_t)c.v[i];
    out[4 * i + 1] = (uint8_t)(c.v[i] >> 8);
    out[4 * i + 2] = (uint8_t)(c.v[i] >> 16);
    out[4 * i + 3] = (uint8_t)(c.v[i] >> 24);
  }
}

__device__ __forceinline__ G1A g1_affine_with(const G1J& p, const Fp& inv_zz_zzz) {
  if (p.is_inf()) return G1A::inf();
  return {f_mul(p.X, f_mul(inv_zz_zzz, p.ZZZ)), f_mul(p.Y, f_mul(inv_zz_zzz, p.ZZ))};
}

// Canonical affine encoding of one G1 point (64 bytes: x, y; infinity as zeros); one thread.
__device__ __forceinline__ void encode_g1(const G1J& P, uint8_t* out) {
  const Fp inv = P.is_inf() ? Fp::one() : f_inv(f_mul(P.ZZ, P.ZZZ));
  const G1A q = g1_affine_with(P, inv);
  write_canon(out, q.x);
  write_canon(out + 32, q.y);
}

// Canonical encodings of A (bytes 0..63) and C (192..255) with one shared inversion
// (Montgomery's trick); one thread.
__device__ __forceinline__ void encode_a_c(const G1J& A, const G1J& C, uint8_t* proof) {
  Fp za = A.is_inf() ? Fp::one() : f_mul(A.ZZ, A.ZZZ);
  Fp zc = C.is_inf() ? Fp::one() : f_mul(C.ZZ, C.ZZZ);
  Fp inv = f_inv(f_mul(za, zc));
  G1A a = g1_affine_with(A, f_mul(inv, zc));
  G1A c = g1_affine_with(C, f_mul(inv, za));
  write_canon(proof + 0, a.x);
  write_canon(proof + 32, a.y);
  write_canon(proof + 192, c.x);
  write_canon(proof + 224, c.y);
}

// Canonical encoding of B (bytes 64..191: x.c0, x.c1, y.c0, y.c1); one thread.
__device__ __forceinline__ void encode_b(const G2J& B, uint8_t* proof) {
  G2A q = p_to_affine(B);
  write_canon(proof + 64, q.x.c0);
  write_canon(proof + 96, q.x.c1);
  write_canon(proof + 128, q.y.c0);
  write_canon(proof + 160, q.y.c1);
}

}  // namespace zkvc
