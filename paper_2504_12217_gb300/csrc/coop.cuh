// Point additions and doublings spread over a quad of four lanes.
//
// One thread doing an XYZZ addition runs its 14 Montgomery products back to back, and a
// product costs a lone thread about 1,300 cycles (the multiply issue rate of one warp):
// a lone thread needs about 9 us per G1 addition.  Where few sums remain (the upper levels of the bucket-sum trees, the 2^b
// scalings, the window combination) that latency, not throughput, sets the time.  The
// formulas have independent products: add-2008-s has four rounds of at most four
// independent products, dbl-2008-s-1 three.  So four lanes hold the same operands, each
// computes one product of a round, and the products are broadcast with warp shuffles
// before the products that depend on them; all four lanes end with the same result.
//
// Every lane of a quad must call these functions with the same operands (the branches on
// infinity and on equal x are then uniform within the quad).  The shuffles name only the
// quad's own lanes, so quads of one warp may take different paths.
#pragma once
#include "curve.cuh"

namespace zkvc {

__device__ __forceinline__ int quad_lane() { return threadIdx.x & 3; }
__device__ __forceinline__ int quad_base() { return (threadIdx.x & 31) & ~3; }
__device__ __forceinline__ unsigned quad_mask() { return 0xFu << quad_base(); }

// lane `src` of the quad's value of x, in every lane of the quad
template <class T>
__device__ __forceinline__ T quad_bcast(const T& x, int src) {
  static_assert(sizeof(T) % 4 == 0, "32-bit words");
  T r;
  const uint32_t* s = reinterpret_cast<const uint32_t*>(&x);
  uint32_t* d = reinterpret_cast<uint32_t*>(&r);
  const unsigned m = quad_mask();
  const int lane = quad_base() + src;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); i++) d[i] = __shfl_sync(m, s[i], lane);
  return r;
}

// a_k for quad lane k.  The choice is made with bit masks, not a conditional: a chain of
// conditionals lets the compiler sink the product that consumes the operand into per-lane
// branches, and the quad then runs its four products one after another instead of side
// by side (measured: a round of pick + product took twice a product's latency).
template <class T>
__device__ __forceinline__ T quad_pick(const T& a0, const T& a1, const T& a2, const T& a3) {
  const int k = quad_lane();
  const uint32_t m0 = 0u - uint32_t(k == 0), m1 = 0u - uint32_t(k == 1), m2 = 0u - uint32_t(k == 2),
                 m3 = 0u - uint32_t(k == 3);
  T r;
  const uint32_t* w0 = reinterpret_cast<const uint32_t*>(&a0);
  const uint32_t* w1 = reinterpret_cast<const uint32_t*>(&a1);
  const uint32_t* w2 = reinterpret_cast<const uint32_t*>(&a2);
  const uint32_t* w3 = reinterpret_cast<const uint32_t*>(&a3);
  uint32_t* d = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); i++) d[i] = (w0[i] & m0) | (w1[i] & m1) | (w2[i] & m2) | (w3[i] & m3);
  return r;
}

// dbl-2008-s-1 in three product rounds:
//   (V = U^2, X^2)  ->  (W = U V, S = X V, M^2, ZZ3 = V ZZ)  ->  (M (S - X3), W Y, ZZZ3 = W ZZZ)
template <class F>
__device__ __forceinline__ XYZZ<F> p_dbl_quad_body(const XYZZ<F>& p) {
  if (p.is_inf() || p.Y.is_zero()) return XYZZ<F>::inf();
  const F U = f_dbl(p.Y);
  F m = f_mulx(quad_pick(U, p.X, U, p.X), quad_pick(U, p.X, U, p.X));
  const F V = quad_bcast(m, 0), X2 = quad_bcast(m, 1);
  const F M = f_add(f_dbl(X2), X2);
  m = f_mulx(quad_pick(U, p.X, M, V), quad_pick(V, V, M, p.ZZ));
  const F W = quad_bcast(m, 0), S = quad_bcast(m, 1), MM = quad_bcast(m, 2), ZZ3 = quad_bcast(m, 3);
  const F X3 = f_sub(MM, f_dbl(S));
  const F SX = f_sub(S, X3);
  m = f_mulx(quad_pick(M, W, W, M), quad_pick(SX, p.Y, p.ZZZ, SX));
  const F Y3 = f_sub(quad_bcast(m, 0), quad_bcast(m, 1));
  const F ZZZ3 = quad_bcast(m, 2);
  return {X3, Y3, ZZ3, ZZZ3};
}

// add-2008-s in four product rounds:
//   (U1, U2, S1, S2)  ->  (PP = P^2, R^2, ZZ1 ZZ2, ZZZ1 ZZZ2)  ->  (PPP = P PP, Q = U1 PP,
//   ZZ3 = ZZ1 ZZ2 PP)  ->  (R (Q - X3), S1 PPP, ZZZ3 = ZZZ1 ZZZ2 PPP)
template <class F>
__device__ __forceinline__ XYZZ<F> p_add_quad_body(const XYZZ<F>& p, const XYZZ<F>& q) {
  if (q.is_inf()) return p;
  if (p.is_inf()) return q;
  F m = f_mulx(quad_pick(p.X, q.X, p.Y, q.Y), quad_pick(q.ZZ, p.ZZ, q.ZZZ, p.ZZZ));
  const F U1 = quad_bcast(m, 0), U2 = quad_bcast(m, 1), S1 = quad_bcast(m, 2), S2 = quad_bcast(m, 3);
  const F P = f_sub(U2, U1), R = f_sub(S2, S1);
  if (P.is_zero()) {
    if (R.is_zero()) return p_dbl_quad_body(p);
    return XYZZ<F>::inf();
  }
  m = f_mulx(quad_pick(P, R, p.ZZ, p.ZZZ), quad_pick(P, R, q.ZZ, q.ZZZ));
  const F PP = quad_bcast(m, 0), RR = quad_bcast(m, 1), Z2 = quad_bcast(m, 2), Z3 = quad_bcast(m, 3);
  m = f_mulx(quad_pick(P, U1, Z2, P), PP);
  const F PPP = quad_bcast(m, 0), Q = quad_bcast(m, 1), ZZ3 = quad_bcast(m, 2);
  const F X3 = f_sub(f_sub(RR, PPP), f_dbl(Q));
  const F QX = f_sub(Q, X3);
  m = f_mulx(quad_pick(R, S1, Z3, R), quad_pick(QX, PPP, PPP, QX));
  const F Y3 = f_sub(quad_bcast(m, 0), quad_bcast(m, 1));
  const F ZZZ3 = quad_bcast(m, 2);
  return {X3, Y3, ZZ3, ZZZ3};
}

// madd-2008-s (XYZZ + affine) in four product rounds:
//   (U2 = X2 ZZ1, S2 = Y2 ZZZ1)  ->  (PP = P^2, R^2)  ->  (PPP = P PP, Q = X1 PP, ZZ3 = ZZ1 PP)
//   ->  (R (Q - X3), Y1 PPP, ZZZ3 = ZZZ1 PPP)
template <class F>
__device__ __forceinline__ XYZZ<F> p_add_affine_quad_body(const XYZZ<F>& p, const Affine<F>& q) {
  if (q.is_inf()) return p;
  if (p.is_inf()) return XYZZ<F>::from_affine(q);
  F m = f_mulx(quad_pick(q.x, q.y, q.x, q.y), quad_pick(p.ZZ, p.ZZZ, p.ZZ, p.ZZZ));
  const F P = f_sub(quad_bcast(m, 0), p.X), R = f_sub(quad_bcast(m, 1), p.Y);
  if (P.is_zero()) {
    if (R.is_zero()) return p_dbl_affine(q);  // rare: every lane doubles alone
    return XYZZ<F>::inf();
  }
  m = f_mulx(quad_pick(P, R, P, R), quad_pick(P, R, P, R));
  const F PP = quad_bcast(m, 0), RR = quad_bcast(m, 1);
  m = f_mulx(quad_pick(P, p.X, p.ZZ, P), PP);
  const F PPP = quad_bcast(m, 0), Q = quad_bcast(m, 1), ZZ3 = quad_bcast(m, 2);
  const F X3 = f_sub(f_sub(RR, PPP), f_dbl(Q));
  const F QX = f_sub(Q, X3);
  m = f_mulx(quad_pick(R, p.Y, p.ZZZ, R), quad_pick(QX, PPP, PPP, QX));
  const F Y3 = f_sub(quad_bcast(m, 0), quad_bcast(m, 1));
  const F ZZZ3 = quad_bcast(m, 2);
  return {X3, Y3, ZZ3, ZZZ3};
}

static __device__ __noinline__ G1J p_add_affine_quad_g1(G1J p, G1A q) { return p_add_affine_quad_body(p, q); }
static __device__ __noinline__ G2J p_add_affine_quad_g2(G2J p, G2A q) { return p_add_affine_quad_body(p, q); }
__device__ __forceinline__ G1J p_add_affine_quad(const G1J& p, const G1A& q) { return p_add_affine_quad_g1(p, q); }
__device__ __forceinline__ G2J p_add_affine_quad(const G2J& p, const G2A& q) { return p_add_affine_quad_g2(p, q); }

static __device__ __noinline__ G1J p_dbl_quad_g1(G1J p) { return p_dbl_quad_body(p); }
static __device__ __noinline__ G2J p_dbl_quad_g2(G2J p) { return p_dbl_quad_body(p); }
static __device__ __noinline__ G1J p_add_quad_g1(G1J p, G1J q) { return p_add_quad_body(p, q); }
static __device__ __noinline__ G2J p_add_quad_g2(G2J p, G2J q) { return p_add_quad_body(p, q); }

__device__ __forceinline__ G1J p_dbl_quad(const G1J& p) { return p_dbl_quad_g1(p); }

__device__ __forceinline__ G2J p_dbl_quad(const G2J& p) { return p_dbl_quad_g2(p); }
__device__ __forceinline__ G1J p_add_quad(const G1J& p, const G1J& q) { return p_add_quad_g1(p, q); }
__device__ __forceinline__ G2J p_add_quad(const G2J& p, const G2J& q) { return p_add_quad_g2(p, q); }

}  // namespace zkvc
