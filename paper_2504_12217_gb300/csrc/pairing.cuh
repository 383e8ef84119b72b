// Optimal ate pairing over BN254 on the GPU, for Groth16 verification (zkVC Sec. II:
// Verify checks e(A, B) = e(alpha, beta) e(IC(x), gamma) e(C, delta)).
//
// Tower: Fp6 = Fp2[v]/(v^3 - xi), Fp12 = Fp6[w]/(w^2 - v), xi = 9 + i, so w^6 = xi and an
// element is sum_m c_m w^m (c_m in Fp2, m = 2j + k for the coefficient j of v in part k).
// G2 lives on the D-type twist y^2 = x^3 + 3/xi; psi(x, y) = (x w^2, y w^3) maps it into
// E(Fp12).
//
// Miller loop: f_(6u+2, Q)(P) with T on the twist in Jacobian coordinates (no inversions).
// The tangent / chord through T (and Q) evaluated at P is l = yP - lambda xP w +
// (lambda xR - yR) w^3 for a point R on the line; each line is used scaled by a factor in
// Fp2 (2 Y Z^3 for doublings, Z3 for additions), which the final exponentiation removes.
// Two closing additions with pi(Q) and -pi^2(Q) (Frobenius on the twist) complete the
// optimal ate loop; 6u + 2 > 0 for this curve, so no final conjugation.
//
// Final exponentiation f^((p^12 - 1)/r): the easy part f^((p^6 - 1)(p^2 + 1)) with one
// inversion and a Frobenius, then the hard part (p^4 - p^2 + 1)/r = p^3 + l2 p^2 + l1 p + l0
// with l2 = 6u^2 + 1, l1 = -36u^3 - 18u^2 - 12u + 1, l0 = -36u^3 - 30u^2 - 18u - 2 (an
// identity in u checked by the tests), through three exponentiations by u; in the
// cyclotomic subgroup an inverse is a conjugation.  The result is exactly the pairing
// value, not a power of it.
#pragma once
#include "curve.cuh"

namespace zkvc {

struct Fp6 {
  Fp2 c0, c1, c2;
};
struct Fp12 {
  Fp6 c0, c1;
};

// ------------------------------------------------------------------ Fp2 helpers
__device__ __forceinline__ Fp2 f2_conj(const Fp2& a) { return {a.c0, f_neg(a.c1)}; }
__device__ __forceinline__ Fp2 f2_mul_fp(const Fp2& a, const Fp& s) { return {f_mul(a.c0, s), f_mul(a.c1, s)}; }
// (a0 + a1 i)(9 + i) = (9 a0 - a1) + (a0 + 9 a1) i
__device__ __forceinline__ Fp2 f2_mul_xi(const Fp2& a) {
  Fp t0 = f_add(f_dbl(f_dbl(f_dbl(a.c0))), a.c0);
  Fp t1 = f_add(f_dbl(f_dbl(f_dbl(a.c1))), a.c1);
  return {f_sub(t0, a.c1), f_add(a.c0, t1)};
}

// ------------------------------------------------------------------ Fp6
// The out-of-line tower functions take their operands by reference and copy them into
// locals on entry: with a 384-byte by-value Fp12 parameter read again after nested
// out-of-line calls, the exponentiation by u returned wrong values on sm_103a (found
// against the oracle; the same loop inlined into its caller was correct).
__device__ __forceinline__ Fp6 f6_add(const Fp6& a, const Fp6& b) {
  return {f_add(a.c0, b.c0), f_add(a.c1, b.c1), f_add(a.c2, b.c2)};
}
__device__ __forceinline__ Fp6 f6_sub(const Fp6& a, const Fp6& b) {
  return {f_sub(a.c0, b.c0), f_sub(a.c1, b.c1), f_sub(a.c2, b.c2)};
}
__device__ __forceinline__ Fp6 f6_neg(const Fp6& a) { return {f_neg(a.c0), f_neg(a.c1), f_neg(a.c2)}; }
// (c0, c1, c2) v = (xi c2, c0, c1)
__device__ __forceinline__ Fp6 f6_mul_v(const Fp6& a) { return {f2_mul_xi(a.c2), a.c0, a.c1}; }

static __device__ __noinline__ Fp6 f6_mul(const Fp6& a_in, const Fp6& b_in) {
  const Fp6 a = a_in, b = b_in;
  Fp2 t0 = f_mul(a.c0, b.c0), t1 = f_mul(a.c1, b.c1), t2 = f_mul(a.c2, b.c2);
  Fp2 c0 = f_add(t0, f2_mul_xi(f_sub(f_sub(f_mul(f_add(a.c1, a.c2), f_add(b.c1, b.c2)), t1), t2)));
  Fp2 c1 = f_add(f_sub(f_sub(f_mul(f_add(a.c0, a.c1), f_add(b.c0, b.c1)), t0), t1), f2_mul_xi(t2));
  Fp2 c2 = f_add(f_sub(f_sub(f_mul(f_add(a.c0, a.c2), f_add(b.c0, b.c2)), t0), t2), t1);
  return {c0, c1, c2};
}

__device__ __forceinline__ Fp6 f6_inv(const Fp6& a) {
  Fp2 A = f_sub(f_sqr(a.c0), f2_mul_xi(f_mul(a.c1, a.c2)));
  Fp2 B = f_sub(f2_mul_xi(f_sqr(a.c2)), f_mul(a.c0, a.c1));
  Fp2 C = f_sub(f_sqr(a.c1), f_mul(a.c0, a.c2));
  Fp2 F = f_add(f_mul(a.c0, A), f2_mul_xi(f_add(f_mul(a.c2, B), f_mul(a.c1, C))));
  Fp2 fi = f_inv(F);
  return {f_mul(A, fi), f_mul(B, fi), f_mul(C, fi)};
}

// ------------------------------------------------------------------ Fp12
__device__ __forceinline__ Fp12 f12_one() {
  Fp12 r;
  r.c0 = {Fp2::one(), Fp2::zero(), Fp2::zero()};
  r.c1 = {Fp2::zero(), Fp2::zero(), Fp2::zero()};
  return r;
}

static __device__ __noinline__ Fp12 f12_mul(const Fp12& a_in, const Fp12& b_in) {
  const Fp12 a = a_in, b = b_in;
  Fp6 t0 = f6_mul(a.c0, b.c0), t1 = f6_mul(a.c1, b.c1);
  Fp12 r;
  r.c0 = f6_add(t0, f6_mul_v(t1));
  r.c1 = f6_sub(f6_sub(f6_mul(f6_add(a.c0, a.c1), f6_add(b.c0, b.c1)), t0), t1);
  return r;
}

// (a0 + a1 w)^2 = (a0 + a1)(a0 + v a1) - t - v t + 2 t w, t = a0 a1
static __device__ __noinline__ Fp12 f12_sqr(const Fp12& a_in) {
  const Fp12 a = a_in;
  Fp6 t = f6_mul(a.c0, a.c1);
  Fp12 r;
  r.c0 = f6_sub(f6_sub(f6_mul(f6_add(a.c0, a.c1), f6_add(a.c0, f6_mul_v(a.c1))), t), f6_mul_v(t));
  r.c1 = f6_add(t, t);
  return r;
}

__device__ __forceinline__ Fp12 f12_conj(const Fp12& a) { return {a.c0, f6_neg(a.c1)}; }

// (a0 + a1 w)^-1 = (a0 - a1 w) / (a0^2 - v a1^2)
__device__ __forceinline__ Fp12 f12_inv(const Fp12& a) {
  Fp6 t = f6_sub(f6_mul(a.c0, a.c0), f6_mul_v(f6_mul(a.c1, a.c1)));
  Fp6 ti = f6_inv(t);
  return {f6_mul(a.c0, ti), f6_neg(f6_mul(a.c1, ti))};
}

__device__ __forceinline__ bool f12_is_one(const Fp12& a) {
  Fp12 o = f12_one();
  return a.c0.c0 == o.c0.c0 && a.c0.c1 == o.c0.c1 && a.c0.c2 == o.c0.c2 && a.c1.c0 == o.c1.c0 &&
         a.c1.c1 == o.c1.c1 && a.c1.c2 == o.c1.c2;
}

// Frobenius constants: gam[k][m] = xi^(m (p^k - 1) / 6) for k = 1, 2, 3 and m < 6 (index k-1).
struct FrobTab {
  Fp2 g[3][6];
};

// f^(p^k): c_m -> c_m^(p^k) gam[k][m] with c^(p^k) = conj(c) for odd k
__device__ __forceinline__ Fp12 f12_frob(const Fp12& a, const FrobTab& T, int k) {
  const Fp2* g = T.g[k - 1];
  const bool cj = (k & 1) != 0;
  auto tw = [&](const Fp2& c, int m) { return f_mul(cj ? f2_conj(c) : c, g[m]); };
  Fp12 r;
  r.c0 = {tw(a.c0.c0, 0), tw(a.c0.c1, 2), tw(a.c0.c2, 4)};
  r.c1 = {tw(a.c1.c0, 1), tw(a.c1.c1, 3), tw(a.c1.c2, 5)};
  return r;
}

// ------------------------------------------------------------------ Miller loop
struct G2Jac {
  Fp2 X, Y, Z;
};

// l = l0 + l1 w + l3 w^3 = (l0, 0, 0) + (l1, l3, 0) w
__device__ __forceinline__ Fp12 line_to_f12(const Fp2& l0, const Fp2& l1, const Fp2& l3) {
  Fp12 r;
  r.c0 = {l0, Fp2::zero(), Fp2::zero()};
  r.c1 = {l1, l3, Fp2::zero()};
  return r;
}

// tangent at T evaluated at P (scaled by 2 Y Z^3), and T <- 2T
__device__ __forceinline__ Fp12 miller_dbl(G2Jac& T, const Fp& xP, const Fp& yP) {
  Fp2 A = f_sqr(T.X), B = f_sqr(T.Y), C = f_sqr(B);
  Fp2 ZZ = f_sqr(T.Z);
  Fp2 D = f_dbl(f_sub(f_sub(f_sqr(f_add(T.X, B)), A), C));
  Fp2 E = f_add(f_dbl(A), A);
  Fp2 F = f_sqr(E);
  Fp2 l3 = f_sub(f_mul(E, T.X), f_dbl(B));   // 3 X^3 - 2 Y^2
  Fp2 X3 = f_sub(F, f_dbl(D));
  Fp2 Y3 = f_sub(f_mul(E, f_sub(D, X3)), f_dbl(f_dbl(f_dbl(C))));
  Fp2 Z3 = f_dbl(f_mul(T.Y, T.Z));
  Fp2 l0 = f2_mul_fp(f_mul(Z3, ZZ), yP);     // 2 Y Z^3 yP
  Fp2 l1 = f_neg(f2_mul_fp(f_mul(E, ZZ), xP));  // -3 X^2 Z^2 xP
  T = {X3, Y3, Z3};
  return line_to_f12(l0, l1, l3);
}

// chord through T and Q (affine) evaluated at P (scaled by Z3), and T <- T + Q
__device__ __forceinline__ Fp12 miller_add(G2Jac& T, const G2A& Q, const Fp& xP, const Fp& yP) {
  Fp2 ZZ = f_sqr(T.Z), ZZZ = f_mul(T.Z, ZZ);
  Fp2 H = f_sub(f_mul(Q.x, ZZ), T.X);
  Fp2 R = f_sub(f_mul(Q.y, ZZZ), T.Y);
  Fp2 HH = f_sqr(H), HHH = f_mul(H, HH), V = f_mul(T.X, HH);
  Fp2 X3 = f_sub(f_sub(f_sqr(R), HHH), f_dbl(V));
  Fp2 Y3 = f_sub(f_mul(R, f_sub(V, X3)), f_mul(T.Y, HHH));
  Fp2 Z3 = f_mul(T.Z, H);
  Fp2 l0 = f2_mul_fp(Z3, yP);
  Fp2 l1 = f_neg(f2_mul_fp(R, xP));
  Fp2 l3 = f_sub(f_mul(R, Q.x), f_mul(Z3, Q.y));
  T = {X3, Y3, Z3};
  return line_to_f12(l0, l1, l3);
}

static constexpr uint64_t BN_U = 4965661367192848881ull;  // the curve parameter u

// bit i of the loop scalar 6u + 2 (65 bits; bit 64 is set, the low 64 bits wrap)
__device__ __forceinline__ bool ate_bit(int i) {
  const uint64_t lo = 6ull * BN_U + 2ull;
  return i == 64 ? true : ((lo >> i) & 1ull) != 0;
}

// f_(6u+2, Q)(P) with the two Frobenius additions; P, Q affine (Montgomery), not infinity
static __device__ __noinline__ Fp12 miller_loop(const G1A& P_in, const G2A& Q_in, const FrobTab& T) {
  const G1A P = P_in;
  const G2A Q = Q_in;
  Fp12 f = f12_one();
  if (P.is_inf() || Q.is_inf()) return f;
  G2Jac R{Q.x, Q.y, Fp2::one()};
  for (int i = 63; i >= 0; i--) {
    f = f12_mul(f12_sqr(f), miller_dbl(R, P.x, P.y));
    if (ate_bit(i)) f = f12_mul(f, miller_add(R, Q, P.x, P.y));
  }
  // pi(Q) = (conj(x) xi^((p-1)/3), conj(y) xi^((p-1)/2)); pi^2(Q) = (x xi^((p^2-1)/3), y xi^((p^2-1)/2))
  G2A Q1{f_mul(f2_conj(Q.x), T.g[0][2]), f_mul(f2_conj(Q.y), T.g[0][3])};
  G2A Q2n{f_mul(Q.x, T.g[1][2]), f_neg(f_mul(Q.y, T.g[1][3]))};
  f = f12_mul(f, miller_add(R, Q1, P.x, P.y));
  f = f12_mul(f, miller_add(R, Q2n, P.x, P.y));
  return f;
}

// ------------------------------------------------------------------ final exponentiation
static __device__ __noinline__ Fp12 f12_pow_u(const Fp12& a_in) {  // a^u
  const Fp12 a = a_in;
  const uint64_t u = BN_U;
  Fp12 r = a;
  for (int i = 61; i >= 0; i--) {  // u has 63 bits: top bit 62
    r = f12_sqr(r);
    if ((u >> i) & 1ull) r = f12_mul(r, a);
  }
  return r;
}

static __device__ __noinline__ Fp12 final_exp(const Fp12& f_in, const FrobTab& T) {
  const Fp12 f = f_in;
  // easy part: f^(p^6 - 1) = conj(f) / f, then ^(p^2 + 1)
  Fp12 t = f12_mul(f12_conj(f), f12_inv(f));
  t = f12_mul(f12_frob(t, T, 2), t);
  // hard part
  Fp12 a = f12_pow_u(t), b = f12_pow_u(a), c = f12_pow_u(b);  // t^u, t^u^2, t^u^3
  Fp12 t2 = f12_sqr(t);
  Fp12 a2 = f12_sqr(a), a3 = f12_mul(a2, a), a6 = f12_sqr(a3), a12 = f12_sqr(a6), a18 = f12_mul(a12, a6);
  Fp12 b2 = f12_sqr(b), b3 = f12_mul(b2, b), b6 = f12_sqr(b3), b12 = f12_sqr(b6), b18 = f12_mul(b12, b6);
  Fp12 b30 = f12_mul(b18, b12);
  Fp12 c2 = f12_sqr(c), c4 = f12_sqr(c2), c8 = f12_sqr(c4), c9 = f12_mul(c8, c), c18 = f12_sqr(c9), c36 = f12_sqr(c18);
  Fp12 y0 = f12_conj(f12_mul(f12_mul(c36, b30), f12_mul(a18, t2)));  // t^l0
  Fp12 y1 = f12_mul(f12_conj(f12_mul(f12_mul(c36, b18), a12)), t);   // t^l1
  Fp12 y2 = f12_mul(b6, t);                                          // t^l2
  Fp12 r = f12_mul(f12_frob(t, T, 3), f12_frob(y2, T, 2));
  r = f12_mul(r, f12_frob(y1, T, 1));
  return f12_mul(r, y0);
}

}  // namespace zkvc
