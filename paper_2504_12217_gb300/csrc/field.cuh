// BN254 prime fields on 8 x 32-bit limbs in Montgomery form, and Fp2 = Fp[i]/(i^2 + 1).
//
// The Groth16 prover of zkVC (Sec. IV: libsnark's groth16 backend) works in the scalar
// field Fr (witness, QAP polynomials, NTT) and the base field Fp (curve coordinates).
// Both moduli are below 2^254, which the bounds below rely on.
//
// Multiplication is CIOS Montgomery (coarsely integrated operand scanning): for each
// limb b_i of the multiplier the row t += a * b_i is two carry chains of mad.lo / mad.hi
// (PTX mad.lo.cc / madc.hi.cc, one IMAD each), then m = t_0 * (-N^-1 mod 2^32) and
// t = (t + m N) / 2^32 the same way.  With a, b < N < 2^254 every intermediate stays
// below 2^288, so a 9-word accumulator never carries out and the result is < 2N before
// the single conditional subtraction.  Cost: 4 * 8 * 8 + 8 = 264 IMADs per product.
#pragma once
#include <cstdint>

namespace zkvc {

// ------------------------------------------------------------------ compile-time bignum
struct U256c {
  uint32_t w[8];
};

constexpr U256c cx_dbl_mod(U256c x, U256c m) {
  U256c r{};
  uint32_t c = 0;
  for (int i = 0; i < 8; i++) {
    uint64_t v = ((uint64_t)x.w[i] << 1) | c;
    r.w[i] = (uint32_t)v;
    c = (uint32_t)(v >> 32);
  }
  bool ge = c != 0;
  if (!ge) {
    ge = true;
    for (int i = 7; i >= 0; i--) {
      if (r.w[i] != m.w[i]) {
        ge = r.w[i] > m.w[i];
        break;
      }
    }
  }
  if (ge) {
    uint64_t br = 0;
    for (int i = 0; i < 8; i++) {
      uint64_t v = (uint64_t)r.w[i] - m.w[i] - br;
      r.w[i] = (uint32_t)v;
      br = (v >> 63) & 1;
    }
  }
  return r;
}

constexpr U256c cx_pow2_mod(int k, U256c m) {
  U256c x{};
  x.w[0] = 1;
  for (int i = 0; i < k; i++) x = cx_dbl_mod(x, m);
  return x;
}

constexpr uint32_t cx_neg_inv32(uint32_t m0) {
  uint32_t x = m0;  // Newton iteration for m0^-1 mod 2^32 (m0 odd)
  for (int i = 0; i < 5; i++) x = x * (2u - m0 * x);
  return 0u - x;
}

// ------------------------------------------------------------------ field parameters
// p and r of BN254 (alt_bn128), little-endian 32-bit limbs.
struct FpCfg {
  static constexpr U256c MOD = {{0xd87cfd47u, 0x3c208c16u, 0x6871ca8du, 0x97816a91u,
                                 0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u}};
  static constexpr U256c R1 = cx_pow2_mod(256, MOD);
  static constexpr U256c R2 = cx_pow2_mod(512, MOD);
  static constexpr U256c R3 = cx_pow2_mod(768, MOD);
  static constexpr uint32_t INV = cx_neg_inv32(MOD.w[0]);
};

struct FrCfg {
  static constexpr U256c MOD = {{0xf0000001u, 0x43e1f593u, 0x79b97091u, 0x2833e848u,
                                 0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u}};
  static constexpr U256c R1 = cx_pow2_mod(256, MOD);
  static constexpr U256c R2 = cx_pow2_mod(512, MOD);
  static constexpr U256c R3 = cx_pow2_mod(768, MOD);
  static constexpr uint32_t INV = cx_neg_inv32(MOD.w[0]);
};

#define ZKVC_LIMB_SWITCH(ARR, i)                                               \
  switch (i) {                                                                 \
    case 0: return ARR.w[0];                                                   \
    case 1: return ARR.w[1];                                                   \
    case 2: return ARR.w[2];                                                   \
    case 3: return ARR.w[3];                                                   \
    case 4: return ARR.w[4];                                                   \
    case 5: return ARR.w[5];                                                   \
    case 6: return ARR.w[6];                                                   \
    default: return ARR.w[7];                                                  \
  }

template <class C>
__host__ __device__ __forceinline__ constexpr uint32_t mod_limb(int i) { ZKVC_LIMB_SWITCH(C::MOD, i) }
template <class C>
__host__ __device__ __forceinline__ constexpr uint32_t r1_limb(int i) { ZKVC_LIMB_SWITCH(C::R1, i) }
template <class C>
__host__ __device__ __forceinline__ constexpr uint32_t r2_limb(int i) { ZKVC_LIMB_SWITCH(C::R2, i) }
template <class C>
__host__ __device__ __forceinline__ constexpr uint32_t r3_limb(int i) { ZKVC_LIMB_SWITCH(C::R3, i) }

// ------------------------------------------------------------------ carry-chain rows
// t[0..8] += a[0..7] * b : low halves into t[0..7] (carry into t[8]), then high halves
// into t[1..8].  The caller guarantees that the 288-bit sum fits.
__device__ __forceinline__ void mac_row(uint32_t (&t)[9], const uint32_t (&a)[8], uint32_t b) {
  asm("mad.lo.cc.u32  %0, %9,  %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9,  %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]),
        "+r"(t[7]), "+r"(t[8])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
        "r"(b));
}

// r = a + b over 8 limbs; returns the carry out.
__device__ __forceinline__ uint32_t add8(uint32_t (&r)[8], const uint32_t (&a)[8], const uint32_t (&b)[8]) {
  uint32_t c;
  asm("add.cc.u32  %0, %9,  %17;\n\t"
      "addc.cc.u32 %1, %10, %18;\n\t"
      "addc.cc.u32 %2, %11, %19;\n\t"
      "addc.cc.u32 %3, %12, %20;\n\t"
      "addc.cc.u32 %4, %13, %21;\n\t"
      "addc.cc.u32 %5, %14, %22;\n\t"
      "addc.cc.u32 %6, %15, %23;\n\t"
      "addc.cc.u32 %7, %16, %24;\n\t"
      "addc.u32    %8, 0, 0;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(c)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
        "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  return c;
}

// r = a - b over 8 limbs; returns 1 if it borrowed (a < b).
__device__ __forceinline__ uint32_t sub8(uint32_t (&r)[8], const uint32_t (&a)[8], const uint32_t (&b)[8]) {
  uint32_t br;
  asm("sub.cc.u32  %0, %9,  %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32    %8, 0, 0;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(br)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
        "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  return br & 1u;
}

// ------------------------------------------------------------------ prime field element
template <class C>
struct Field {
  uint32_t v[8];

  __device__ __forceinline__ static Field zero() {
    Field r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = 0;
    return r;
  }
  __device__ __forceinline__ static Field one() {  // R mod N (Montgomery form of 1)
    Field r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = r1_limb<C>(i);
    return r;
  }
  __device__ __forceinline__ static Field modulus() {
    Field r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = mod_limb<C>(i);
    return r;
  }
  __device__ __forceinline__ bool is_zero() const {
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc |= v[i];
    return acc == 0;
  }
  __device__ __forceinline__ bool operator==(const Field& o) const {
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc |= v[i] ^ o.v[i];
    return acc == 0;
  }
  __device__ __forceinline__ bool operator!=(const Field& o) const { return !(*this == o); }
};

template <class C>
__device__ __forceinline__ Field<C> f_add(const Field<C>& a, const Field<C>& b) {
  Field<C> s, d;
  add8(s.v, a.v, b.v);  // a + b < 2N < 2^255: no carry out
  const Field<C> m = Field<C>::modulus();
  uint32_t br = sub8(d.v, s.v, m.v);
  return br ? s : d;
}

template <class C>
__device__ __forceinline__ Field<C> f_sub(const Field<C>& a, const Field<C>& b) {
  Field<C> d, e;
  uint32_t br = sub8(d.v, a.v, b.v);
  const Field<C> m = Field<C>::modulus();
  add8(e.v, d.v, m.v);
  return br ? e : d;
}

template <class C>
__device__ __forceinline__ Field<C> f_neg(const Field<C>& a) {
  return f_sub(Field<C>::zero(), a);
}

template <class C>
__device__ __forceinline__ Field<C> f_dbl(const Field<C>& a) { return f_add(a, a); }

// Montgomery product a b R^-1 mod N, CIOS with carry-chain rows (reference form; the
// product-scanning f_mul below is the one the kernels use).
template <class C>
__device__ __forceinline__ Field<C> f_mul_cios(const Field<C>& a, const Field<C>& b) {
  uint32_t t[9];
#pragma unroll
  for (int i = 0; i < 9; i++) t[i] = 0;
  uint32_t m[8];
#pragma unroll
  for (int i = 0; i < 8; i++) m[i] = mod_limb<C>(i);
#pragma unroll
  for (int i = 0; i < 8; i++) {
    mac_row(t, a.v, b.v[i]);
    uint32_t q = t[0] * C::INV;
    mac_row(t, m, q);  // t[0] becomes 0
#pragma unroll
    for (int j = 0; j < 8; j++) t[j] = t[j + 1];
    t[8] = 0;
  }
  Field<C> r, d;
#pragma unroll
  for (int i = 0; i < 8; i++) r.v[i] = t[i];
  uint32_t br = sub8(d.v, r.v, m);
  return br ? r : d;
}

// One term x y of a product-scanning column: (t2, t1, t0) += x y as mad.lo.cc /
// madc.hi.cc / addc.
__device__ __forceinline__ void col_mac(uint32_t& t0, uint32_t& t1, uint32_t& t2, uint32_t x, uint32_t y) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
      : "+r"(t0), "+r"(t1), "+r"(t2)
      : "r"(x), "r"(y));
}

// Montgomery product a b R^-1 mod N by finely integrated product scanning (Koc, Acar and
// Kaliski, "Analyzing and comparing Montgomery multiplication algorithms", 1996): column
// i of the 16-word result sums every a_j b_(i-j) and m_j N_(i-j) into a 96-bit
// accumulator; for i < 8 its low word then fixes m_i = t_0 (-N^-1) mod 2^32 and m_i N_0
// clears it; the columns 8 .. 15 are the result.  A column holds at most 16 products
// below 2^64 plus the carry of the previous one, so 96 bits never overflow; with a, b < N
// the result is below 2N and one conditional subtraction makes it canonical.  Same IMAD
// count as CIOS (264); on GB300 it runs at 18.1 T IMAD-equivalents/s in a throughput
// loop against 12.3-12.6 T/s for the CIOS forms (zkvc_imad_rate forms 5-7): its
// independent low/high word pairs and short carries issue better than CIOS's long
// carry chains.
template <class C>
__device__ __forceinline__ Field<C> f_mul(const Field<C>& a, const Field<C>& b) {
  uint32_t m[8];
  Field<C> r, d;
  uint32_t t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      col_mac(t0, t1, t2, a.v[j], b.v[i - j]);
      col_mac(t0, t1, t2, m[j], mod_limb<C>(i - j));
    }
    col_mac(t0, t1, t2, a.v[i], b.v[0]);
    m[i] = t0 * C::INV;
    col_mac(t0, t1, t2, m[i], mod_limb<C>(0));  // t0 becomes 0
    t0 = t1;
    t1 = t2;
    t2 = 0;
  }
#pragma unroll
  for (int i = 8; i < 15; i++) {
#pragma unroll
    for (int j = i - 7; j < 8; j++) {
      col_mac(t0, t1, t2, a.v[j], b.v[i - j]);
      col_mac(t0, t1, t2, m[j], mod_limb<C>(i - j));
    }
    r.v[i - 8] = t0;
    t0 = t1;
    t1 = t2;
    t2 = 0;
  }
  r.v[7] = t0;  // r < 2N < 2^255: no further word
  const Field<C> mm = Field<C>::modulus();
  const uint32_t br = sub8(d.v, r.v, mm.v);
  return br ? r : d;
}

template <class C>
__device__ __forceinline__ Field<C> f_sqr(const Field<C>& a) { return f_mul(a, a); }

// Out-of-line Montgomery product with 64-bit accumulation: CIOS rows written with
// 32 x 32 + 64-bit multiply-adds in plain C (reference form: 12.6 T IMAD-equivalents/s in
// zkvc_imad_rate form 6, against 18.1 T/s for f_mulc below).
template <class C>
__device__ __noinline__ Field<C> f_mulc_cios(Field<C> a, Field<C> b) {
  uint32_t t[10];
#pragma unroll
  for (int i = 0; i < 10; i++) t[i] = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      uint64_t s = (uint64_t)a.v[j] * b.v[i] + t[j] + c;  // < 2^64
      t[j] = (uint32_t)s;
      c = s >> 32;
    }
    uint64_t s8 = (uint64_t)t[8] + c;
    t[8] = (uint32_t)s8;
    t[9] = (uint32_t)(s8 >> 32);
    uint32_t q = t[0] * C::INV;
    c = ((uint64_t)q * mod_limb<C>(0) + t[0]) >> 32;  // low word cancels
#pragma unroll
    for (int j = 1; j < 8; j++) {
      uint64_t s = (uint64_t)q * mod_limb<C>(j) + t[j] + c;
      t[j - 1] = (uint32_t)s;
      c = s >> 32;
    }
    uint64_t s7 = (uint64_t)t[8] + c;
    t[7] = (uint32_t)s7;
    t[8] = t[9] + (uint32_t)(s7 >> 32);
    t[9] = 0;
  }
  Field<C> r, d;
  uint32_t m[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    r.v[i] = t[i];
    m[i] = mod_limb<C>(i);
  }
  uint32_t br = sub8(d.v, r.v, m);  // result < 2N < 2^255, so t[8] = 0 here
  return br ? r : d;
}

// Out-of-line product-scanning Montgomery product for the point formulas: called, not
// inlined, so that the large formulas keep one copy of the product's ~400 instructions
// (fully inlined point formulas stall on instruction fetch).
template <class C>
__device__ __noinline__ Field<C> f_mulc(Field<C> a, Field<C> b) {
  return f_mul(a, b);
}

template <class C>
__device__ __forceinline__ Field<C> f_to_mont(const Field<C>& a) {
  Field<C> r2;
#pragma unroll
  for (int i = 0; i < 8; i++) r2.v[i] = r2_limb<C>(i);
  return f_mul(a, r2);
}

template <class C>
__device__ __forceinline__ Field<C> f_from_mont(const Field<C>& a) {
  Field<C> one_raw = Field<C>::zero();
  one_raw.v[0] = 1;
  return f_mul(a, one_raw);
}

// Canonical value from a small signed integer (|v| < 2^31), already in Montgomery form.
template <class C>
__device__ __forceinline__ Field<C> f_from_int(int32_t v) {
  Field<C> x = Field<C>::zero();
  uint32_t mag = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;
  x.v[0] = mag;
  x = f_to_mont(x);
  return v < 0 ? f_neg(x) : x;
}

// a^e for an exponent given as 8 limbs (plain square-and-multiply, MSB first).
template <class C>
__device__ __forceinline__ Field<C> f_pow(const Field<C>& a, const uint32_t (&e)[8]) {
  Field<C> r = Field<C>::one();
  for (int i = 7; i >= 0; i--) {
    for (int bit = 31; bit >= 0; bit--) {
      r = f_sqr(r);
      if ((e[i] >> bit) & 1u) r = f_mul(r, a);
    }
  }
  return r;
}

// Inverse of a Montgomery-form element (a R -> a^-1 R); 0 maps to 0.  The integer
// inverse y^-1 mod N of y = a R comes from the binary GCD, and a product with R^3 brings
// y^-1 = a^-1 R^-1 back to Montgomery form.  Not constant-time.
//
// Binary GCD with Bezout coefficients: (a, b) = (y, N), (u, v) = (1, 0), invariants
// a = u y and b = v y (mod N); an odd a larger than b becomes a - b (u - v), a smaller one
// is swapped first; an even a is halved (u halved mod N).  a reaches 0 and b = gcd = 1
// within 2 len(N) - 1 steps, and then v = y^-1.
//
// Fast path (Pornin, "Optimized Binary GCD for Modular Inversion", 2020): 30 steps at a
// time on 62-bit stand-ins for a and b (their low 30 bits and top 32 bits at the common
// length n = max(len a, len b, 62)), whose parity and order decisions are recorded as an
// integer matrix [[f0, g0], [f1, g1]] with entries at most 2^30 in magnitude; then the
// exact update (a, b) <- ((f0 a + g0 b) / 2^30, (f1 a + g1 b) / 2^30), made non-negative
// by flipping a row's sign, and (u, v) <- the same rows applied to (u, v) and divided by
// 2^30 mod N (one Montgomery step), which keeps the invariants without a final
// power-of-two correction.  ceil((2 * 254 - 1) / 30) = 17 rounds reach a = 0, b = 1 for
// 254-bit moduli; a round after that leaves (a, b, v) unchanged.  Should the check at the
// end ever fail, the one-step-at-a-time loop below recomputes the inverse.  (One thread:
// about 50 k cycles against 78 k for the one-step loop.)
__device__ __forceinline__ void shr1_8(uint32_t (&x)[8], uint32_t top) {
#pragma unroll
  for (int i = 0; i < 7; i++) x[i] = (x[i] >> 1) | (x[i + 1] << 31);
  x[7] = (x[7] >> 1) | (top << 31);
}

__device__ __forceinline__ bool is_one8(const uint32_t (&x)[8]) {
  uint32_t acc = x[0] ^ 1u;
#pragma unroll
  for (int i = 1; i < 8; i++) acc |= x[i];
  return acc == 0;
}


namespace bgcd {
// bit length of x | y
__device__ __forceinline__ int len2(const uint32_t (&x)[8], const uint32_t (&y)[8]) {
  int n = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint32_t w = x[i] | y[i];
    n = w ? 32 * i + 32 - __clz(w) : n;
  }
  return n;
}

// (x mod 2^30) + 2^30 floor(x / 2^(n - 32)) for len(x) <= n, 62 <= n <= 256
__device__ __forceinline__ uint64_t approx(const uint32_t (&x)[8], int n) {
  const int s = n - 32, q = s >> 5, r = s & 31;
  uint32_t lo = 0, hi = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    lo = i == q ? x[i] : lo;
    hi = i == q + 1 ? x[i] : hi;
  }
  const uint64_t top = ((((uint64_t)hi << 32) | lo) >> r) & 0xffffffffull;
  return (uint64_t)(x[0] & 0x3fffffffu) | (top << 30);
}

// t = x f + y g as a 9-limb two's complement number (x, y < 2^254, |f|, |g| <= 2^30):
// x f is x |f| with every limb complemented and 1 added when f < 0
__device__ __forceinline__ void lin9(uint32_t (&t)[9], const uint32_t (&x)[8], int32_t f, const uint32_t (&y)[8],
                                     int32_t g) {
  const uint32_t mf = (uint32_t)(f < 0 ? -f : f), mg = (uint32_t)(g < 0 ? -g : g);
  const uint32_t sf = (uint32_t)(f >> 31), sg = (uint32_t)(g >> 31);
  uint64_t cf = 0, cg = 0, c = (sf & 1u) + (sg & 1u);
#pragma unroll
  for (int i = 0; i < 9; i++) {
    if (i < 8) {
      cf += (uint64_t)x[i] * mf;
      cg += (uint64_t)y[i] * mg;
    }
    c += (uint64_t)((uint32_t)cf ^ sf) + ((uint32_t)cg ^ sg);
    t[i] = (uint32_t)c;
    c >>= 32;
    cf >>= 32;
    cg >>= 32;
  }
}

// t >>= 30, arithmetic
__device__ __forceinline__ void sar30(uint32_t (&t)[9]) {
#pragma unroll
  for (int i = 0; i < 8; i++) t[i] = (t[i] >> 30) | (t[i + 1] << 2);
  t[8] = (uint32_t)((int32_t)t[8] >> 30);
}

// t = -t when s = ~0 (s = 0: unchanged)
__device__ __forceinline__ void cneg9(uint32_t (&t)[9], uint32_t s) {
  uint64_t c = s & 1u;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    c += (uint32_t)(t[i] ^ s);
    t[i] = (uint32_t)c;
    c >>= 32;
  }
}

// t += m, or t -= m, over 9 limbs
__device__ __forceinline__ void addm9(uint32_t (&t)[9], const uint32_t (&m)[8], bool sub) {
  const uint32_t x = sub ? 0xffffffffu : 0u;
  uint64_t c = sub ? 1u : 0u;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    c += (uint64_t)t[i] + ((i < 8 ? m[i] : 0u) ^ x);
    t[i] = (uint32_t)c;
    c >>= 32;
  }
}

// (x f + y g) / 2^30 mod m in [0, m), for x, y in [0, m): q = t (-m^-1) mod 2^30 makes
// t + q m divisible by 2^30, and -2m < (t + q m) / 2^30 < 3m
__device__ __forceinline__ void upd_mod(uint32_t (&out)[8], const uint32_t (&x)[8], int32_t f, const uint32_t (&y)[8],
                                        int32_t g, const uint32_t (&m)[8], uint32_t minv) {
  uint32_t t[9];
  lin9(t, x, f, y, g);
  const uint32_t q = (t[0] * minv) & 0x3fffffffu;
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    if (i < 8) c += (uint64_t)m[i] * q;
    c += t[i];
    t[i] = (uint32_t)c;
    c >>= 32;
  }
  sar30(t);
  for (int k = 0; k < 2 && (int32_t)t[8] < 0; k++) addm9(t, m, false);
  for (int k = 0; k < 2; k++) {
    uint32_t d9[9];
#pragma unroll
    for (int i = 0; i < 9; i++) d9[i] = t[i];
    addm9(d9, m, true);
    if ((int32_t)d9[8] < 0) break;
#pragma unroll
    for (int i = 0; i < 9; i++) t[i] = d9[i];
  }
#pragma unroll
  for (int i = 0; i < 8; i++) out[i] = t[i];
}
}  // namespace bgcd

// y^-1 mod N for 0 < y < N (integers, 8 limbs); false if the rounds did not finish
template <class C>
__device__ __noinline__ bool inv_bgcd(const uint32_t (&y)[8], uint32_t (&out)[8]) {
  uint32_t a[8], b[8], u[8], v[8], m[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    m[i] = mod_limb<C>(i);
    a[i] = y[i];
    b[i] = m[i];
    u[i] = i == 0;
    v[i] = 0;
  }
  const uint32_t minv = C::INV;  // -N^-1 mod 2^32, hence also mod 2^30
  for (int round = 0; round < 17; round++) {
    const int n = max(bgcd::len2(a, b), 62);
    uint64_t ab = bgcd::approx(a, n), bb = bgcd::approx(b, n);
    int32_t f0 = 1, g0 = 0, f1 = 0, g1 = 1;
    // 30 binary-GCD steps on the stand-ins, without branches
#pragma unroll 10
    for (int j = 0; j < 30; j++) {
      const bool odd = ab & 1u;
      const bool sw = odd && ab < bb;
      const uint64_t na = sw ? bb : ab, nb = sw ? ab : bb;
      const int32_t nf0 = sw ? f1 : f0, ng0 = sw ? g1 : g0, nf1 = sw ? f0 : f1, ng1 = sw ? g0 : g1;
      ab = (odd ? na - nb : na) >> 1;
      bb = nb;
      f0 = odd ? nf0 - nf1 : nf0;
      g0 = odd ? ng0 - ng1 : ng0;
      f1 = nf1 * 2;
      g1 = ng1 * 2;
    }
    uint32_t ta[9], tb[9];
    bgcd::lin9(ta, a, f0, b, g0);
    bgcd::lin9(tb, a, f1, b, g1);
    bgcd::sar30(ta);
    bgcd::sar30(tb);
    const uint32_t sa = (uint32_t)((int32_t)ta[8] >> 31), sb = (uint32_t)((int32_t)tb[8] >> 31);
    bgcd::cneg9(ta, sa);
    bgcd::cneg9(tb, sb);
    f0 = sa ? -f0 : f0;
    g0 = sa ? -g0 : g0;
    f1 = sb ? -f1 : f1;
    g1 = sb ? -g1 : g1;
    uint32_t nu[8], nv[8];
    bgcd::upd_mod(nu, u, f0, v, g0, m, minv);
    bgcd::upd_mod(nv, u, f1, v, g1, m, minv);
#pragma unroll
    for (int i = 0; i < 8; i++) {
      a[i] = ta[i];
      b[i] = tb[i];
      u[i] = nu[i];
      v[i] = nv[i];
    }
  }
  uint32_t z = b[0] ^ 1u;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    z |= a[i] | (i ? b[i] : 0u);
    out[i] = v[i];
  }
  return z == 0;
}

template <class C>
__device__ __noinline__ Field<C> f_inv(const Field<C>& a) {
  if (a.is_zero()) return Field<C>::zero();
  {
    uint32_t r[8];
    if (inv_bgcd<C>(a.v, r)) {
      Field<C> x, r3;
#pragma unroll
      for (int i = 0; i < 8; i++) {
        x.v[i] = r[i];
        r3.v[i] = r3_limb<C>(i);
      }
      return f_mul(x, r3);
    }
  }
  uint32_t p[8], u[8], v[8], x1[8], x2[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    p[i] = mod_limb<C>(i);
    u[i] = a.v[i];
    v[i] = p[i];
    x1[i] = 0;
    x2[i] = 0;
  }
  x1[0] = 1;
  while (!is_one8(u) && !is_one8(v)) {
    while ((u[0] & 1u) == 0) {
      shr1_8(u, 0);
      if (x1[0] & 1u) {
        uint32_t c = add8(x1, x1, p);
        shr1_8(x1, c);
      } else {
        shr1_8(x1, 0);
      }
    }
    while ((v[0] & 1u) == 0) {
      shr1_8(v, 0);
      if (x2[0] & 1u) {
        uint32_t c = add8(x2, x2, p);
        shr1_8(x2, c);
      } else {
        shr1_8(x2, 0);
      }
    }
    uint32_t d[8];
    if (!sub8(d, u, v)) {  // u >= v
#pragma unroll
      for (int i = 0; i < 8; i++) u[i] = d[i];
      if (sub8(d, x1, x2)) add8(d, d, p);
#pragma unroll
      for (int i = 0; i < 8; i++) x1[i] = d[i];
    } else {
      sub8(d, v, u);
#pragma unroll
      for (int i = 0; i < 8; i++) v[i] = d[i];
      if (sub8(d, x2, x1)) add8(d, d, p);
#pragma unroll
      for (int i = 0; i < 8; i++) x2[i] = d[i];
    }
  }
  Field<C> r, r3;
  const bool uone = is_one8(u);
#pragma unroll
  for (int i = 0; i < 8; i++) {
    r.v[i] = uone ? x1[i] : x2[i];
    r3.v[i] = r3_limb<C>(i);
  }
  return f_mul(r, r3);
}

using Fp = Field<FpCfg>;
using Fr = Field<FrCfg>;

// ------------------------------------------------------------------ Fp2 = Fp[i]/(i^2+1)
struct Fp2 {
  Fp c0, c1;
  __device__ __forceinline__ static Fp2 zero() { return {Fp::zero(), Fp::zero()}; }
  __device__ __forceinline__ static Fp2 one() { return {Fp::one(), Fp::zero()}; }
  __device__ __forceinline__ bool is_zero() const { return c0.is_zero() && c1.is_zero(); }
  __device__ __forceinline__ bool operator==(const Fp2& o) const { return c0 == o.c0 && c1 == o.c1; }
  __device__ __forceinline__ bool operator!=(const Fp2& o) const { return !(*this == o); }
};

__device__ __forceinline__ Fp2 f_add(const Fp2& a, const Fp2& b) { return {f_add(a.c0, b.c0), f_add(a.c1, b.c1)}; }
__device__ __forceinline__ Fp2 f_sub(const Fp2& a, const Fp2& b) { return {f_sub(a.c0, b.c0), f_sub(a.c1, b.c1)}; }
__device__ __forceinline__ Fp2 f_neg(const Fp2& a) { return {f_neg(a.c0), f_neg(a.c1)}; }
__device__ __forceinline__ Fp2 f_dbl(const Fp2& a) { return {f_dbl(a.c0), f_dbl(a.c1)}; }

// Karatsuba: (a0 + a1 i)(b0 + b1 i) = (a0 b0 - a1 b1) + ((a0 + a1)(b0 + b1) - a0 b0 - a1 b1) i
// (out of line, on the compact Fp product: G2 formulas call it ~14 times each)
static __device__ __noinline__ Fp2 f_mul(Fp2 a, Fp2 b) {
  Fp t0 = f_mulc(a.c0, b.c0);
  Fp t1 = f_mulc(a.c1, b.c1);
  Fp t2 = f_mulc(f_add(a.c0, a.c1), f_add(b.c0, b.c1));
  return {f_sub(t0, t1), f_sub(f_sub(t2, t0), t1)};
}

// (a0 + a1 i)^2 = (a0 + a1)(a0 - a1) + 2 a0 a1 i
static __device__ __noinline__ Fp2 f_sqr(Fp2 a) {
  Fp t = f_mulc(a.c0, a.c1);
  return {f_mulc(f_add(a.c0, a.c1), f_sub(a.c0, a.c1)), f_dbl(t)};
}

__device__ __forceinline__ Fp2 f_inv(const Fp2& a) {
  Fp n = f_add(f_sqr(a.c0), f_sqr(a.c1));
  Fp ni = f_inv(n);
  return {f_mul(a.c0, ni), f_neg(f_mul(a.c1, ni))};
}

__device__ __forceinline__ Fp2 f_to_mont(const Fp2& a) { return {f_to_mont(a.c0), f_to_mont(a.c1)}; }
__device__ __forceinline__ Fp2 f_from_mont(const Fp2& a) { return {f_from_mont(a.c0), f_from_mont(a.c1)}; }

// ------------------------------------------------------------------ memory helpers
template <class F>
__device__ __forceinline__ F ld_field(const F* p) {
  static_assert(sizeof(F) % 16 == 0, "16-byte vector loads");
  F r;
  uint32_t* d = reinterpret_cast<uint32_t*>(&r);
  const uint4* s = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(F) / 16); i++) {
    uint4 q = s[i];
    d[4 * i] = q.x;
    d[4 * i + 1] = q.y;
    d[4 * i + 2] = q.z;
    d[4 * i + 3] = q.w;
  }
  return r;
}

template <class F>
__device__ __forceinline__ void st_field(F* p, const F& x) {
  uint4* d = reinterpret_cast<uint4*>(p);
  const uint32_t* s = reinterpret_cast<const uint32_t*>(&x);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(F) / 16); i++) d[i] = make_uint4(s[4 * i], s[4 * i + 1], s[4 * i + 2], s[4 * i + 3]);
}

}  // namespace zkvc
