// G1 arithmetic with the limbs of every field element spread over eight lanes.
//
// A lone thread's Montgomery product is limited by the multiply issue rate of its warp
// (about 1,300 cycles whatever the active-lane count), which makes serial chains of point
// operations slow (a scalar multiplication is about 250 doublings in a row).  Here lane j
// of an eight-lane group holds limb j (32 bits) of a field element, and the group computes
// one CIOS Montgomery product cooperatively: each lane does one column of every row, so a
// product costs the group 16 multiply-adds per lane instead of 264 in one lane.
//
// The product (operand scanning, rows i = 0..7, in every lane j of the group):
//   u_j = a_i b_j + t_j + c1_j;   m = lo(position 0) * (-p^-1 mod 2^32);
//   v_j = m p_j + lo(u_j) + c2_j;  c1_j = hi(u_j), c2_j = hi(v_j);  t_j = lo(v_(j+1)).
// lo(v_0) = 0 by the choice of m, so the shift t_j <- lo(v_(j+1)) is the division by 2^32;
// the carries hi(u_j), hi(v_j) belong one position up and stay in lane j after the shift.
// Every bound fits 64 bits: a_i b_j + t + c1 and m p_j + lo(u) + c2 are at most 2^64 - 1.
// The row's m needs position 0 only: every lane tracks lane 0's carries itself and gets
// lo(v_1) by one broadcast, so m is computed locally and one row costs one shuffle round
// trip plus two dependent multiplies.  After eight rows the value sum (t_j + c1_j + c2_j)
// 2^(32 j) is the CIOS result, below 2p, brought to canonical limbs by one shift of the
// small carries and one carry-lookahead.
//
// Carry-lookahead over the eight limbs: each lane has a generate bit (its limb overflows
// by itself) and a propagate bit (its limb overflows iff a carry comes in), never both.
// With G and P the group's bytes of two warp ballots, the carries into the limbs are the
// carry bits of the binary sum (G | P) + G, i.e. ((G | P) + G) xor P, and bit 8 of the
// sum is the carry out.  Additions, subtractions and the conditional subtraction of p all
// use it.
//
// A warp holds four groups.  The point formulas (XYZZ, as in curve.cuh) run their
// products in rounds of up to four independent products: group g computes product g of
// a round and the results are broadcast to the other groups by one shuffle per product.
// Every lane of a warp must call these functions together with the same operands (the
// ballots name the whole warp, and the branches on infinity are then warp-uniform).
#pragma once
#include "curve.cuh"

namespace zkvc {

constexpr unsigned SL_FULL = 0xffffffffu;

__device__ __forceinline__ int sl_limb() { return threadIdx.x & 7; }
__device__ __forceinline__ int sl_group() { return (threadIdx.x >> 3) & 3; }
__device__ __forceinline__ int sl_base() { return threadIdx.x & 24; }

// this lane's limb of p and of R mod p (Montgomery one)
__device__ __forceinline__ uint32_t sl_p() {
  const int j = sl_limb();
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) r |= mod_limb<FpCfg>(i) & (0u - uint32_t(j == i));
  return r;
}
__device__ __forceinline__ uint32_t sl_one() {
  const int j = sl_limb();
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) r |= r1_limb<FpCfg>(i) & (0u - uint32_t(j == i));
  return r;
}

struct SlCarry {
  uint32_t in, out;  // carry into this lane's limb; carry out of limb 7
};

__device__ __forceinline__ SlCarry sl_carry(bool gen, bool prop) {
  const int sh = sl_base();
  const uint32_t G = (__ballot_sync(SL_FULL, gen) >> sh) & 0xffu;
  const uint32_t P = (__ballot_sync(SL_FULL, prop) >> sh) & 0xffu;
  const uint32_t S = (G | P) + G;
  return {((S ^ P) >> sl_limb()) & 1u, (S >> 8) & 1u};
}

__device__ __forceinline__ bool sl_is_zero(uint32_t x) {
  return ((__ballot_sync(SL_FULL, x != 0) >> sl_base()) & 0xffu) == 0;
}

// x < 2p  ->  x mod p
__device__ __forceinline__ uint32_t sl_reduce(uint32_t x, uint32_t pj) {
  const SlCarry b = sl_carry(x < pj, x == pj);
  return b.out ? x : x - pj - b.in;
}

__device__ __forceinline__ uint32_t sl_add(uint32_t a, uint32_t b) {
  const uint64_t s = (uint64_t)a + b;  // a + b < 2p < 2^255: no carry out of limb 7
  const uint32_t x = (uint32_t)s;
  const SlCarry c = sl_carry((s >> 32) != 0, x == 0xffffffffu);
  return sl_reduce(x + c.in, sl_p());
}

__device__ __forceinline__ uint32_t sl_sub(uint32_t a, uint32_t b) {
  const SlCarry bw = sl_carry(a < b, a == b);
  const uint32_t x = a - b - bw.in;
  const uint64_t s = (uint64_t)x + (bw.out ? sl_p() : 0u);  // a < b: add p back
  const uint32_t y = (uint32_t)s;
  const SlCarry c = sl_carry((s >> 32) != 0, y == 0xffffffffu);
  return y + c.in;
}

__device__ __forceinline__ uint32_t sl_neg(uint32_t a) { return sl_sub(0u, a); }

// Montgomery product a b R^-1 mod p, a and b canonical; result canonical
__device__ __forceinline__ uint32_t sl_mul(uint32_t a, uint32_t b) {
  const int j = sl_limb(), base = sl_base();
  const uint32_t pj = sl_p(), p0 = mod_limb<FpCfg>(0), inv = FpCfg::INV;
  uint32_t ai[8];
#pragma unroll
  for (int i = 0; i < 8; i++) ai[i] = __shfl_sync(SL_FULL, a, base + i);
  const uint32_t b0 = __shfl_sync(SL_FULL, b, base);
  uint32_t t = 0, c1 = 0, c2 = 0;   // this lane's position
  uint32_t t0 = 0, d1 = 0, d2 = 0;  // position 0 (lane 0's t, c1, c2)
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint64_t pre = (uint64_t)ai[i] * b + c1;
    const uint64_t pre0 = (uint64_t)ai[i] * b0 + d1;
    const uint32_t k = ((uint32_t)pre0 + d2) * inv;
    const uint32_t m = t0 * inv + k;  // lo(a_i b_0 + t_0 + c1_0 + c2_0) * inv
    const uint64_t u = pre + t, u0 = pre0 + t0;
    const uint64_t v = (uint64_t)m * pj + ((uint64_t)(uint32_t)u + c2);
    const uint64_t v0 = (uint64_t)m * p0 + ((uint64_t)(uint32_t)u0 + d2);
    c1 = (uint32_t)(u >> 32);
    c2 = (uint32_t)(v >> 32);
    d1 = (uint32_t)(u0 >> 32);
    d2 = (uint32_t)(v0 >> 32);
    const uint32_t lo = (uint32_t)v;
    const uint32_t dn = __shfl_down_sync(SL_FULL, lo, 1, 8);
    t = j == 7 ? 0u : dn;
    t0 = __shfl_sync(SL_FULL, lo, base + 1);
  }
  // sum (t + c1 + c2) 2^(32 j) < 2p: move each position's small carry (<= 2) up one
  // limb, then one lookahead for the ripple that can remain
  const uint64_t s = (uint64_t)t + c1 + c2;
  const uint32_t up = __shfl_up_sync(SL_FULL, (uint32_t)(s >> 32), 1, 8);
  const uint64_t y = (uint64_t)(uint32_t)s + (j == 0 ? 0u : up);
  const uint32_t x = (uint32_t)y;
  const SlCarry c = sl_carry((y >> 32) != 0, x == 0xffffffffu);
  return sl_reduce(x + c.in, pj);
}

// ------------------------------------------------------------------ points (G1, XYZZ)
struct SlG1 {
  uint32_t X, Y, ZZ, ZZZ;
};

__device__ __forceinline__ SlG1 sl_inf() {
  const uint32_t one = sl_one();
  return {one, one, 0u, 0u};
}

// this lane's limbs of a G1J in global or shared memory; only group 0 stores
__device__ __forceinline__ SlG1 sl_ld(const G1J* p) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(p);
  const int j = sl_limb();
  return {w[j], w[8 + j], w[16 + j], w[24 + j]};
}
__device__ __forceinline__ void sl_st(G1J* p, const SlG1& x) {
  if (sl_group() != 0) return;
  uint32_t* w = reinterpret_cast<uint32_t*>(p);
  const int j = sl_limb();
  w[j] = x.X;
  w[8 + j] = x.Y;
  w[16 + j] = x.ZZ;
  w[24 + j] = x.ZZZ;
}

// operand k for group k (bit masks, not conditionals: see quad_pick in coop.cuh)
__device__ __forceinline__ uint32_t sl_pick(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3) {
  const int g = sl_group();
  return (a0 & (0u - uint32_t(g == 0))) | (a1 & (0u - uint32_t(g == 1))) | (a2 & (0u - uint32_t(g == 2))) |
         (a3 & (0u - uint32_t(g == 3)));
}
// group k's product, in every group
__device__ __forceinline__ uint32_t sl_from(uint32_t m, int k) {
  return __shfl_sync(SL_FULL, m, 8 * k + sl_limb());
}

// dbl-2008-s-1 (U = 2Y, V = U^2, W = U V, S = X V, M = 3 X^2, X3 = M^2 - 2S,
// Y3 = M (S - X3) - W Y, ZZ3 = V ZZ, ZZZ3 = W ZZZ) in three product rounds with four
// levels of additions and subtractions (an addition costs two ballot round trips here):
// 2X and 3X come first, so that M = X (3X), 2S = (2X) V and 3S = (3X) V are products, and
// X3 = M^2 - 2S and S - X3 = 3S - M^2 are one level.
//   (V = U^2, M = X 3X)  ->  (W = U V, M^2, 2S, 3S)  ->  (M (S - X3), W Y, W ZZZ, V ZZ)
static __device__ __noinline__ SlG1 sl_pdbl(SlG1 p) {
  const bool inf = sl_is_zero(p.ZZ), y0 = sl_is_zero(p.Y);
  if (inf || y0) return sl_inf();
  const uint32_t U = sl_add(p.Y, p.Y), X2 = sl_add(p.X, p.X);
  const uint32_t X3x = sl_add(X2, p.X);
  uint32_t m = sl_mul(sl_pick(U, p.X, U, p.X), sl_pick(U, X3x, U, X3x));
  const uint32_t V = sl_from(m, 0), M = sl_from(m, 1);
  m = sl_mul(sl_pick(U, M, X2, X3x), sl_pick(V, M, V, V));
  const uint32_t W = sl_from(m, 0), MM = sl_from(m, 1), S2 = sl_from(m, 2), S3 = sl_from(m, 3);
  const uint32_t X3 = sl_sub(MM, S2), SX = sl_sub(S3, MM);
  m = sl_mul(sl_pick(M, W, W, V), sl_pick(SX, p.Y, p.ZZZ, p.ZZ));
  const uint32_t Y3 = sl_sub(sl_from(m, 0), sl_from(m, 1));
  return {X3, Y3, sl_from(m, 3), sl_from(m, 2)};
}

// add-2008-s (U1 = X1 ZZ2, U2 = X2 ZZ1, S1 = Y1 ZZZ2, S2 = Y2 ZZZ1, P = U2 - U1,
// R = S2 - S1, PP = P^2, PPP = P PP, Q = U1 PP, X3 = R^2 - PPP - 2Q, Y3 = R (Q - X3) -
// S1 PPP, ZZ3 = ZZ1 ZZ2 PP, ZZZ3 = ZZZ1 ZZZ2 PPP) in four product rounds with four
// levels of additions and subtractions: the third round's free product gives 2Q =
// (2 U1) PP, so that X3 = (R^2 - PPP) - 2Q and Q - X3 = 3Q - (R^2 - PPP) are one level
// after R^2 - PPP and 3Q.
//   (U1, U2, S1, S2)  ->  (P^2, R^2, ZZ1 ZZ2, ZZZ1 ZZZ2)  ->  (PPP, Q, ZZ3, 2Q)
//   ->  (R (Q - X3), S1 PPP, ZZZ3)
static __device__ __noinline__ SlG1 sl_padd(SlG1 p, SlG1 q) {
  const bool qi = sl_is_zero(q.ZZ), pi = sl_is_zero(p.ZZ);
  if (qi) return p;
  if (pi) return q;
  uint32_t m = sl_mul(sl_pick(p.X, q.X, p.Y, q.Y), sl_pick(q.ZZ, p.ZZ, q.ZZZ, p.ZZZ));
  const uint32_t U1 = sl_from(m, 0), U2 = sl_from(m, 1), S1 = sl_from(m, 2), S2 = sl_from(m, 3);
  const uint32_t P = sl_sub(U2, U1), R = sl_sub(S2, S1), U1x2 = sl_add(U1, U1);
  const bool p0 = sl_is_zero(P), r0 = sl_is_zero(R);
  if (p0) {
    if (r0) return sl_pdbl(p);
    return sl_inf();
  }
  m = sl_mul(sl_pick(P, R, p.ZZ, p.ZZZ), sl_pick(P, R, q.ZZ, q.ZZZ));
  const uint32_t PP = sl_from(m, 0), RR = sl_from(m, 1), Z2 = sl_from(m, 2), Z3 = sl_from(m, 3);
  m = sl_mul(sl_pick(P, U1, Z2, U1x2), PP);
  const uint32_t PPP = sl_from(m, 0), Q = sl_from(m, 1), ZZ3 = sl_from(m, 2), Q2 = sl_from(m, 3);
  const uint32_t A = sl_sub(RR, PPP), Q3 = sl_add(Q, Q2);
  const uint32_t X3 = sl_sub(A, Q2), QX = sl_sub(Q3, A);
  m = sl_mul(sl_pick(R, S1, Z3, R), sl_pick(QX, PPP, PPP, QX));
  const uint32_t Y3 = sl_sub(sl_from(m, 0), sl_from(m, 1));
  return {X3, Y3, ZZ3, sl_from(m, 2)};
}

// k P for one half of a GLV-split scalar (|k| < 2^128 with its sign; glv.h) on one warp:
// the 15 multiples of +-P in shared memory T[1..15] (this warp's own table), then 4-bit
// windows from the top: four doublings and at most one addition per window.
template <class Half>
__device__ __forceinline__ SlG1 sl_mul_half(SlG1 P, const Half& h, G1J* T) {
  if (h.neg) P.Y = sl_neg(P.Y);
  SlG1 prev = P;
  sl_st(T + 1, P);
  for (int i = 2; i < 16; i++) {
    prev = sl_padd(prev, P);
    sl_st(T + i, prev);
  }
  __syncwarp();
  SlG1 acc = sl_inf();
  bool started = false;
  for (int w = 31; w >= 0; w--) {
    if (started) {
      acc = sl_pdbl(acc);
      acc = sl_pdbl(acc);
      acc = sl_pdbl(acc);
      acc = sl_pdbl(acc);
    }
    const uint32_t nib = (h.mag[w >> 3] >> ((w & 7) * 4)) & 15u;
    if (nib) {
      const SlG1 t = sl_ld(T + nib);
      acc = started ? sl_padd(acc, t) : t;
      started = true;
    }
  }
  return acc;
}

}  // namespace zkvc
