// Short-Weierstrass groups G1 = E(Fp): y^2 = x^3 + 3 and G2 = E'(Fp2): y^2 = x^3 + 3/(9+i)
// (BN254), in affine and XYZZ coordinates.
//
// Groth16 (zkVC Sec. II / IV) needs sums of many points: the bucket accumulation of the
// multi-scalar multiplications adds affine base points into running sums, so the hot
// formula is the mixed XYZZ + affine addition (madd-2008-s: 8M + 2S).  XYZZ keeps
// (X, Y, ZZ, ZZZ) with x = X/ZZ, y = Y/ZZZ and ZZ^3 = ZZZ^2; ZZ = 0 is the point at
// infinity.  All formulas are for a = 0 and are generic over the coordinate field, so G2
// reuses them over Fp2.  Affine infinity is encoded as x = y = 0 (not on either curve).
#pragma once
#include "field.cuh"

namespace zkvc {

template <class F>
struct Affine {
  F x, y;
  __device__ __forceinline__ bool is_inf() const { return x.is_zero() && y.is_zero(); }
  __device__ __forceinline__ static Affine inf() { return {F::zero(), F::zero()}; }
};

template <class F>
struct XYZZ {
  F X, Y, ZZ, ZZZ;
  __device__ __forceinline__ bool is_inf() const { return ZZ.is_zero(); }
  __device__ __forceinline__ static XYZZ inf() { return {F::one(), F::one(), F::zero(), F::zero()}; }
  __device__ __forceinline__ static XYZZ from_affine(const Affine<F>& a) {
    if (a.is_inf()) return inf();
    return {a.x, a.y, F::one(), F::one()};
  }
};

using G1A = Affine<Fp>;
using G2A = Affine<Fp2>;
using G1J = XYZZ<Fp>;
using G2J = XYZZ<Fp2>;

// Products used by the point formulas: the compact (rolled, out-of-line) Montgomery
// product.  Smaller code avoids instruction-fetch stalls, which dominate these large
// formulas on GB300: the bucket-accumulation loop runs at 3.7 G mixed additions/s with
// compact products against 2.9 G/s fully unrolled, and the chained XYZZ addition takes
// 10.5 us instead of 12.9 us.
__device__ __forceinline__ Fp f_mulx(const Fp& a, const Fp& b) { return f_mulc(a, b); }
__device__ __forceinline__ Fp f_sqrx(const Fp& a) { return f_mulc(a, a); }
__device__ __forceinline__ Fp2 f_mulx(const Fp2& a, const Fp2& b) { return f_mul(a, b); }
__device__ __forceinline__ Fp2 f_sqrx(const Fp2& a) { return f_sqr(a); }

template <class F>
__device__ __forceinline__ Affine<F> p_neg(const Affine<F>& a) {
  if (a.is_inf()) return a;
  return {a.x, f_neg(a.y)};
}

template <class F>
__device__ __forceinline__ XYZZ<F> p_neg(const XYZZ<F>& a) {
  return {a.X, f_neg(a.Y), a.ZZ, a.ZZZ};
}

// dbl-2008-s-1 (a = 0): U = 2Y, V = U^2, W = U V, S = X V, M = 3 X^2,
// X3 = M^2 - 2S, Y3 = M (S - X3) - W Y, ZZ3 = V ZZ, ZZZ3 = W ZZZ.
template <class F>
__device__ __forceinline__ XYZZ<F> p_dbl_body(const XYZZ<F>& p) {
  if (p.is_inf() || p.Y.is_zero()) return XYZZ<F>::inf();
  F U = f_dbl(p.Y);
  F V = f_sqrx(U);
  F W = f_mulx(U, V);
  F S = f_mulx(p.X, V);
  F X2 = f_sqrx(p.X);
  F M = f_add(f_dbl(X2), X2);
  F X3 = f_sub(f_sqrx(M), f_dbl(S));
  F Y3 = f_sub(f_mulx(M, f_sub(S, X3)), f_mulx(W, p.Y));
  return {X3, Y3, f_mulx(V, p.ZZ), f_mulx(W, p.ZZZ)};
}

// mdbl-2008-s-1: doubling of an affine point into XYZZ.
template <class F>
__device__ __forceinline__ XYZZ<F> p_dbl_affine(const Affine<F>& a) {
  if (a.is_inf() || a.y.is_zero()) return XYZZ<F>::inf();
  F U = f_dbl(a.y);
  F V = f_sqr(U);
  F W = f_mul(U, V);
  F S = f_mul(a.x, V);
  F X2 = f_sqr(a.x);
  F M = f_add(f_dbl(X2), X2);
  F X3 = f_sub(f_sqr(M), f_dbl(S));
  F Y3 = f_sub(f_mul(M, f_sub(S, X3)), f_mul(W, a.y));
  return {X3, Y3, V, W};
}

// madd-2008-s: XYZZ + affine.
template <class F>
__device__ __forceinline__ XYZZ<F> p_add_affine_body(const XYZZ<F>& p, const Affine<F>& q) {
  if (q.is_inf()) return p;
  if (p.is_inf()) return XYZZ<F>::from_affine(q);
  F U2 = f_mulx(q.x, p.ZZ);
  F S2 = f_mulx(q.y, p.ZZZ);
  F P = f_sub(U2, p.X);
  F R = f_sub(S2, p.Y);
  if (P.is_zero()) {
    if (R.is_zero()) return p_dbl_affine(q);
    return XYZZ<F>::inf();
  }
  F PP = f_sqrx(P);
  F PPP = f_mulx(P, PP);
  F Q = f_mulx(p.X, PP);
  F X3 = f_sub(f_sub(f_sqrx(R), PPP), f_dbl(Q));
  F Y3 = f_sub(f_mulx(R, f_sub(Q, X3)), f_mulx(p.Y, PPP));
  return {X3, Y3, f_mulx(p.ZZ, PP), f_mulx(p.ZZZ, PPP)};
}

// add-2008-s: XYZZ + XYZZ.
template <class F>
__device__ __forceinline__ XYZZ<F> p_add_body(const XYZZ<F>& p, const XYZZ<F>& q) {
  if (q.is_inf()) return p;
  if (p.is_inf()) return q;
  F U1 = f_mulx(p.X, q.ZZ);
  F U2 = f_mulx(q.X, p.ZZ);
  F S1 = f_mulx(p.Y, q.ZZZ);
  F S2 = f_mulx(q.Y, p.ZZZ);
  F P = f_sub(U2, U1);
  F R = f_sub(S2, S1);
  if (P.is_zero()) {
    if (R.is_zero()) return p_dbl_body(p);
    return XYZZ<F>::inf();
  }
  F PP = f_sqrx(P);
  F PPP = f_mulx(P, PP);
  F Q = f_mulx(U1, PP);
  F X3 = f_sub(f_sub(f_sqrx(R), PPP), f_dbl(Q));
  F Y3 = f_sub(f_mulx(R, f_sub(Q, X3)), f_mulx(S1, PPP));
  return {X3, Y3, f_mulx(f_mulx(p.ZZ, q.ZZ), PP), f_mulx(f_mulx(p.ZZZ, q.ZZZ), PPP)};
}

// Out-of-line instances: the full additions and doublings, and every G2 operation, are
// called rather than inlined (one copy of ~14 Montgomery products per function instead
// of one per call site); only the G1 mixed addition of the bucket loop is inlined.
static __device__ __noinline__ G1J p_dbl_g1(G1J p) { return p_dbl_body(p); }
static __device__ __noinline__ G2J p_dbl_g2(G2J p) { return p_dbl_body(p); }
static __device__ __noinline__ G1J p_add_g1(G1J p, G1J q) { return p_add_body(p, q); }
static __device__ __noinline__ G2J p_add_g2(G2J p, G2J q) { return p_add_body(p, q); }
static __device__ __noinline__ G2J p_add_affine_g2(G2J p, G2A q) { return p_add_affine_body(p, q); }

__device__ __forceinline__ G1J p_dbl(const G1J& p) { return p_dbl_g1(p); }
__device__ __forceinline__ G2J p_dbl(const G2J& p) { return p_dbl_g2(p); }
__device__ __forceinline__ G1J p_add(const G1J& p, const G1J& q) { return p_add_g1(p, q); }
__device__ __forceinline__ G2J p_add(const G2J& p, const G2J& q) { return p_add_g2(p, q); }
__device__ __forceinline__ G1J p_add_affine(const G1J& p, const G1A& q) { return p_add_affine_body(p, q); }
__device__ __forceinline__ G2J p_add_affine(const G2J& p, const G2A& q) { return p_add_affine_g2(p, q); }

// x = X / ZZ, y = Y / ZZZ with one inversion of ZZ * ZZZ.
template <class F>
__device__ __forceinline__ Affine<F> p_to_affine(const XYZZ<F>& p) {
  if (p.is_inf()) return Affine<F>::inf();
  F inv = f_inv(f_mul(p.ZZ, p.ZZZ));
  F izz = f_mul(inv, p.ZZZ);   // 1/ZZ
  F izzz = f_mul(inv, p.ZZ);   // 1/ZZZ
  return {f_mul(p.X, izz), f_mul(p.Y, izzz)};
}

// Variable-base scalar multiplication with fixed 4-bit windows: a table of the 15
// multiples, then per window four doublings and at most one addition (254 doublings and
// <= 64 additions for a 254-bit scalar instead of double-and-add's ~127 additions).
template <class F>
__device__ __noinline__ XYZZ<F> p_mul_scalar_w4(const XYZZ<F>& p, const uint32_t (&k)[8]) {
  XYZZ<F> T[16];
  T[0] = XYZZ<F>::inf();
  T[1] = p;
  for (int i = 2; i < 16; i++) T[i] = p_add(T[i - 1], p);
  XYZZ<F> acc = XYZZ<F>::inf();
  for (int w = 63; w >= 0; w--) {
    if (w != 63) {
      acc = p_dbl(acc);
      acc = p_dbl(acc);
      acc = p_dbl(acc);
      acc = p_dbl(acc);
    }
    const uint32_t nib = (k[w >> 3] >> ((w & 7) * 4)) & 15u;
    if (nib) acc = p_add(acc, T[nib]);
  }
  return acc;
}

// Curve coefficient b in Montgomery form (runtime conversion of small constants).
__device__ __forceinline__ Fp g1_b() {
  Fp b = Fp::zero();
  b.v[0] = 3;
  return f_to_mont(b);
}

// b' = 3 / (9 + i)
__device__ __forceinline__ Fp2 g2_b() {
  Fp2 xi = Fp2::zero();
  xi.c0.v[0] = 9;
  xi.c1.v[0] = 1;
  Fp2 three = Fp2::zero();
  three.c0.v[0] = 3;
  return f_mul(f_to_mont(three), f_inv(f_to_mont(xi)));
}

template <class F>
__device__ __forceinline__ bool p_on_curve(const Affine<F>& a, const F& b) {
  if (a.is_inf()) return true;
  F lhs = f_sqr(a.y);
  F rhs = f_add(f_mul(f_sqr(a.x), a.x), b);
  return lhs == rhs;
}

// Generators in canonical form: G1 = (1, 2); G2 as published with EIP-197.
__device__ __forceinline__ G1A g1_generator() {
  Fp x = Fp::zero(), y = Fp::zero();
  x.v[0] = 1;
  y.v[0] = 2;
  return {f_to_mont(x), f_to_mont(y)};
}

__device__ __forceinline__ G2A g2_generator() {
  const uint32_t L[4][8] = {
      {0xd992f6edu, 0x46debd5cu, 0xf75edaddu, 0x674322d4u, 0x5e5c4479u, 0x426a0066u, 0x121f1e76u, 0x1800deefu},
      {0xaef312c2u, 0x97e485b7u, 0x35a9e712u, 0xf1aa4933u, 0x31fb5d25u, 0x7260bfb7u, 0x920d483au, 0x198e9393u},
      {0x66fa7daau, 0x4ce6cc01u, 0x0c43d37bu, 0xe3d1e769u, 0x8dcb408fu, 0x4aab7180u, 0xdb8c6debu, 0x12c85ea5u},
      {0xd122975bu, 0x55acdadcu, 0x70b38ef3u, 0xbc4b3133u, 0x690c3395u, 0xec9e99adu, 0x585ff075u, 0x090689d0u}};
  Fp v[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
#pragma unroll
    for (int i = 0; i < 8; i++) v[j].v[i] = L[j][i];
    v[j] = f_to_mont(v[j]);
  }
  return {{v[0], v[1]}, {v[2], v[3]}};
}

}  // namespace zkvc
