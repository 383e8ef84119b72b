// GLV split of a scalar for G1 of BN254 (host side).
//
// G1 has the endomorphism phi(x, y) = (beta x, y), beta a primitive cube root of unity in
// Fp, acting as multiplication by lambda, a cube root of unity mod r, on the order-r
// group.  A scalar k < r is written k = k1 + k2 lambda (mod r) with |k1|, |k2| < 2^127
// by rounding against the short lattice basis v1 = (a1, -b1), v2 = (a2, b2) of
// {(x, y) : x + y lambda = 0 mod r} (Gallant-Lambert-Vanstone, CRYPTO 2001):
//   c1 = floor(k g1 / 2^256), c2 = floor(k g2 / 2^256),
//     g1 = floor(2^256 b2 / r), g2 = floor(2^256 b1 / r),
//   k1 = k - c1 a1 - c2 a2,  k2 = c1 b1 - c2 b2.
// k1 + k2 lambda = k - c1 (a1 - b1 lambda) - c2 (a2 + b2 lambda) = k (mod r) for any
// c1, c2; the rounding keeps both halves short.  Then k P = k1 P + k2 phi(P): two
// 127-bit scalar multiplications that can run side by side.
//
// The constants were derived with the extended Euclidean algorithm on (r, lambda) and
// are checked by a CPU test (the basis spans the lattice, phi(G) = lambda G on the curve,
// and the split reproduces k with short halves).
#pragma once
#include <cstdint>

namespace zkvc {

// lambda = 0xb3c4d79d41a917585bfc41088d8daaa78b17ea66b99c90dd (mod r), and the matching
// beta (mod p), canonical little-endian 32-bit limbs
__host__ __device__ constexpr uint32_t glv_beta_limb(int i) {
  return i == 0 ? 0x77fffffeu : i == 1 ? 0x57634731u : i == 2 ? 0xacdb5c4fu : i == 3 ? 0xd4f263f1u
       : i == 4 ? 0xa0d48bacu : i == 5 ? 0x59e26bceu : 0u;
}
constexpr uint64_t GLV_A1 = 0x89d3256894d213e3ull;                                // a1
constexpr uint64_t GLV_B1[2] = {0x8211bbeb7d4f1128ull, 0x6f4d8248eeb859fcull};     // b1
constexpr uint64_t GLV_A2[2] = {0x0be4e1541221250bull, 0x6f4d8248eeb859fdull};     // a2
constexpr uint64_t GLV_B2 = 0x89d3256894d213e3ull;                                // b2
constexpr uint64_t GLV_G1[2] = {0xd91d232ec7e0b3d7ull, 0x2ull};                  // g1
constexpr uint64_t GLV_G2[3] = {0x7a7bd9d4391eb18dull, 0x4ccef014a773d2cfull, 0x2ull};  // g2

// G2 has the endomorphism psi = (twist)^-1 o Frobenius o twist: for the D-type twist
// y^2 = x^3 + 3/xi (xi = 9 + i) it is psi(x, y) = (conj(x) gx, conj(y) gy) with
// gx = xi^((p-1)/3) and gy = xi^((p-1)/2) in Fp2, and on the order-r subgroup it acts as
// multiplication by lambda2 = p mod r = 6 u^2 (a 127-bit number close to sqrt(r)).  A
// scalar k < r therefore splits as k = k1 + k2 lambda2 with k2 = floor(k / lambda2) and
// k1 = k mod lambda2, both non-negative and below 2^127 (k2 <= (r - 1) / lambda2 =
// 6u^2 + 6u + 3).  The quotient is k g / 2^256 (g = floor(2^256 / lambda2)), low by at
// most one, then corrected.  Checked by a CPU test against the oracle's G2 arithmetic.
constexpr uint64_t PSI_LAMBDA[2] = {0xf83e9682e87cfd46ull, 0x6f4d8248eeb859fbull};  // 6 u^2
constexpr uint64_t PSI_G[3] = {0x2cb62031c8e01941ull, 0x4ccef014a773d2d5ull, 0x2ull};  // floor(2^256 / (6 u^2))
// gx (c = 0: real part, 1: imaginary part), canonical little-endian 32-bit limbs
__host__ __device__ constexpr uint32_t psi_gx_limb(int c, int i) {
  constexpr uint32_t v[2][8] = {
      {0x176f553du, 0x99e39557u, 0xc2c3330cu, 0xb78cc310u, 0xf559b143u, 0x4c0bec3cu, 0x4f7911f7u, 0x2fb34798u},
      {0x640fcba2u, 0x1665d51cu, 0x0b7c9dceu, 0x32ae2a1du, 0xd75a0794u, 0x4ba4cc8bu, 0x61ebae20u, 0x16c9e550u}};
  return v[c][i];
}
// gy
__host__ __device__ constexpr uint32_t psi_gy_limb(int c, int i) {
  constexpr uint32_t v[2][8] = {
      {0x71a0135au, 0xdc540146u, 0xa9c95998u, 0xdbaae0edu, 0xb6e2f9b9u, 0xdc5ec698u, 0x489af5dcu, 0x063cf305u},
      {0x2623b0e3u, 0x82d37f63u, 0x8fa25bd2u, 0x21807dc9u, 0xec796f2bu, 0x0704b5a7u, 0xac41049au, 0x07c03cbcu}};
  return v[c][i];
}

// One half of a split scalar: |k_i| as four 32-bit limbs and its sign.
struct GlvHalf {
  uint32_t mag[4];
  uint32_t neg;
};
struct GlvScalar {
  GlvHalf h[2];  // k1, k2
};

namespace glv_detail {
using u128 = unsigned __int128;

// floor(k * g / 2^256) for k of 4 limbs and g of ng limbs (result fits 2 limbs)
inline void mul_shift256(const uint64_t k[4], const uint64_t* g, int ng, uint64_t out[2]) {
  uint64_t t[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 4; i++) {
    uint64_t carry = 0;
    for (int j = 0; j < ng; j++) {
      u128 s = (u128)k[i] * g[j] + t[i + j] + carry;
      t[i + j] = (uint64_t)s;
      carry = (uint64_t)(s >> 64);
    }
    t[i + ng] += carry;
  }
  out[0] = t[4];
  out[1] = t[5];
}

// r = x * y mod 2^192 (x, y of nx, ny limbs)
inline void mul192(const uint64_t* x, int nx, const uint64_t* y, int ny, uint64_t r[3]) {
  uint64_t t[3] = {0, 0, 0};
  for (int i = 0; i < nx && i < 3; i++) {
    uint64_t carry = 0;
    for (int j = 0; i + j < 3 && j < ny; j++) {
      u128 s = (u128)x[i] * y[j] + t[i + j] + carry;
      t[i + j] = (uint64_t)s;
      carry = (uint64_t)(s >> 64);
    }
    if (i + ny < 3) t[i + ny] += carry;
  }
  r[0] = t[0];
  r[1] = t[1];
  r[2] = t[2];
}

inline void sub192(uint64_t a[3], const uint64_t b[3]) {
  u128 borrow = 0;
  for (int i = 0; i < 3; i++) {
    u128 d = (u128)a[i] - b[i] - borrow;
    a[i] = (uint64_t)d;
    borrow = (d >> 64) ? 1 : 0;
  }
}

inline GlvHalf to_half(uint64_t v[3]) {
  GlvHalf h;
  h.neg = (uint32_t)(v[2] >> 63);
  if (h.neg) {  // magnitude of the two's-complement value
    uint64_t z[3] = {0, 0, 0};
    sub192(z, v);
    v[0] = z[0];
    v[1] = z[1];
    v[2] = z[2];
  }
  h.mag[0] = (uint32_t)v[0];
  h.mag[1] = (uint32_t)(v[0] >> 32);
  h.mag[2] = (uint32_t)v[1];
  h.mag[3] = (uint32_t)(v[1] >> 32);
  return h;
}
}  // namespace glv_detail

// k: 32 bytes little-endian, k < r.  (For larger input the split is still exact mod r
// but the halves may exceed 128 bits; callers check k < r on the device.)
inline GlvScalar glv_split(const uint8_t* k_le) {
  using namespace glv_detail;
  uint64_t k[4];
  for (int i = 0; i < 4; i++) {
    uint64_t w = 0;
    for (int b = 7; b >= 0; b--) w = (w << 8) | k_le[8 * i + b];
    k[i] = w;
  }
  uint64_t c1[2], c2[2];
  mul_shift256(k, GLV_G1, 2, c1);
  mul_shift256(k, GLV_G2, 3, c2);
  // k1 = k - c1 a1 - c2 a2 (mod 2^192)
  uint64_t k1[3] = {k[0], k[1], k[2]}, t[3];
  mul192(c1, 2, &GLV_A1, 1, t);
  sub192(k1, t);
  mul192(c2, 2, GLV_A2, 2, t);
  sub192(k1, t);
  // k2 = c1 b1 - c2 b2 (mod 2^192)
  uint64_t k2[3];
  mul192(c1, 2, GLV_B1, 2, k2);
  mul192(c2, 2, &GLV_B2, 1, t);
  sub192(k2, t);
  GlvScalar g;
  g.h[0] = to_half(k1);
  g.h[1] = to_half(k2);
  return g;
}

#ifdef __CUDACC__
// The same split on the device, for one scalar per thread (the variable-base G1 MSM): the
// halves packed as |k_i| in bits 0..126 of a uint4 and the sign in bit 127 (|k_i| < 2^127).
// k: canonical little-endian 32-bit limbs, k < r.
namespace glv_dev {
// (t, carry) <- t + a b + carry
__device__ __forceinline__ void mac(uint64_t a, uint64_t b, uint64_t& t, uint64_t& carry) {
  uint64_t lo = a * b, hi = __umul64hi(a, b);
  lo += t;
  hi += lo < t;
  lo += carry;
  hi += lo < carry;
  t = lo;
  carry = hi;
}
template <int NG>
__device__ __forceinline__ void mul_shift256(const uint64_t k[4], const uint64_t (&g)[NG], uint64_t out[2]) {
  uint64_t t[4 + NG];
#pragma unroll
  for (int i = 0; i < 4 + NG; i++) t[i] = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < NG; j++) mac(k[i], g[j], t[i + j], carry);
    t[i + NG] = carry;
  }
  out[0] = t[4];
  out[1] = t[5];
}
// r = x y mod 2^192, x of 2 limbs, y of NY limbs
template <int NY>
__device__ __forceinline__ void mul192(const uint64_t x[2], const uint64_t (&y)[NY], uint64_t r[3]) {
  r[0] = r[1] = r[2] = 0;
#pragma unroll
  for (int i = 0; i < 2; i++) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < NY && i + j < 3; j++) mac(x[i], y[j], r[i + j], carry);
    if (i + NY < 3) r[i + NY] += carry;
  }
}
__device__ __forceinline__ void sub192(uint64_t a[3], const uint64_t b[3]) {
  uint64_t borrow = 0;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const uint64_t d = a[i] - b[i], e = d - borrow;
    borrow = (a[i] < b[i]) | (d < borrow);
    a[i] = e;
  }
}
__device__ __forceinline__ uint4 pack(uint64_t v[3]) {
  const uint32_t neg = (uint32_t)(v[2] >> 63);
  if (neg) {
    uint64_t z[3] = {0, 0, 0};
    sub192(z, v);
    v[0] = z[0];
    v[1] = z[1];
  }
  return make_uint4((uint32_t)v[0], (uint32_t)(v[0] >> 32), (uint32_t)v[1],
                    ((uint32_t)(v[1] >> 32) & 0x7fffffffu) | (neg << 31));
}
}  // namespace glv_dev

__device__ __forceinline__ void glv_split_dev(const uint32_t k32[8], uint4* h1, uint4* h2) {
  using namespace glv_dev;
  const uint64_t g1[2] = {GLV_G1[0], GLV_G1[1]}, g2[3] = {GLV_G2[0], GLV_G2[1], GLV_G2[2]};
  const uint64_t a1[1] = {GLV_A1}, a2[2] = {GLV_A2[0], GLV_A2[1]}, b1[2] = {GLV_B1[0], GLV_B1[1]}, b2[1] = {GLV_B2};
  uint64_t k[4];
#pragma unroll
  for (int i = 0; i < 4; i++) k[i] = uint64_t(k32[2 * i]) | (uint64_t(k32[2 * i + 1]) << 32);
  uint64_t c1[2], c2[2], t[3];
  mul_shift256(k, g1, c1);
  mul_shift256(k, g2, c2);
  uint64_t k1[3] = {k[0], k[1], k[2]}, k2[3];  // k1 = k - c1 a1 - c2 a2, k2 = c1 b1 - c2 b2 (mod 2^192)
  mul192(c1, a1, t);
  sub192(k1, t);
  mul192(c2, a2, t);
  sub192(k1, t);
  mul192(c1, b1, k2);
  mul192(c2, b2, t);
  sub192(k2, t);
  *h1 = pack(k1);
  *h2 = pack(k2);
}
// The G2 split k = k1 + k2 lambda2 (both halves non-negative, sign bits 0).
__device__ __forceinline__ void psi_split_dev(const uint32_t k32[8], uint4* h1, uint4* h2) {
  using namespace glv_dev;
  const uint64_t g[3] = {PSI_G[0], PSI_G[1], PSI_G[2]}, lam[2] = {PSI_LAMBDA[0], PSI_LAMBDA[1]};
  uint64_t k[4];
#pragma unroll
  for (int i = 0; i < 4; i++) k[i] = uint64_t(k32[2 * i]) | (uint64_t(k32[2 * i + 1]) << 32);
  uint64_t q[2], t[3];
  mul_shift256(k, g, q);  // floor(k / lambda2) or one less
  uint64_t k1[3] = {k[0], k[1], k[2]};  // k - q lambda2 < 2 lambda2 (mod 2^192)
  mul192(q, lam, t);
  sub192(k1, t);
  const uint64_t lam3[3] = {lam[0], lam[1], 0};
  const bool ge = k1[2] != 0 || k1[1] > lam[1] || (k1[1] == lam[1] && k1[0] >= lam[0]);
  if (ge) {
    sub192(k1, lam3);
    q[0] += 1;
    q[1] += q[0] == 0;
  }
  uint64_t k2[3] = {q[0], q[1], 0};
  *h1 = pack(k1);
  *h2 = pack(k2);
}
#endif

}  // namespace zkvc
