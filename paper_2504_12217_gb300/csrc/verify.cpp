// Groth16 Verify (zkVC Sec. II: Verify decides a proof with the public parameters and the
// public input) on the host: e(A, B) = e(alpha, beta) e(IC(x), gamma) e(C, delta).
//
// Plain C++ with 4 x 64-bit Montgomery limbs (unsigned __int128 products), independent of
// the device code.  The pairing is the optimal ate pairing of BN254:
//   * tower Fp2 = Fp[i]/(i^2 + 1), Fp6 = Fp2[v]/(v^3 - xi), Fp12 = Fp6[w]/(w^2 - v), xi = 9 + i;
//   * G2 lives on the D-type twist y^2 = x^3 + 3/xi; the untwisting map is
//     (x, y) -> (x w^2, y w^3), so a line of slope lam' through T on the twist evaluates at
//     P = (xP, yP) to yP - lam' xP w + (lam' xT - yT) w^3 (a sparse Fp12 element);
//   * Miller loop over the bits of 6u + 2 with affine twist points, then the two lines with
//     pi(Q) and -pi^2(Q), where pi acts on the twist as (conj(x) xi^((p-1)/3), conj(y) xi^((p-1)/2));
//   * final exponentiation f^(p^6 - 1) (conjugate over inverse), then plain
//     square-and-multiply by (p^6 + 1)/r.
// The check multiplies four Miller loops, e(-A, B) e(alpha, beta) e(IC, gamma) e(C, delta),
// and needs one final exponentiation.  Points are validated (canonical coordinates, on
// the curve, B in the order-r subgroup); an invalid point makes the proof invalid.
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/zkvc.h"

namespace zkvc {
void set_error(const char* fmt, ...);
}

namespace {

typedef unsigned __int128 u128;

struct Fq {
  uint64_t v[4];
};

// p = 21888242871839275222246405745257275088696311157297823662689037894645226208583
const uint64_t P[4] = {0x3c208c16d87cfd47ull, 0x97816a916871ca8dull, 0xb85045b68181585dull, 0x30644e72e131a029ull};
// r = 21888242871839275222246405745257275088548364400416034343698204186575808495617
const uint64_t R[4] = {0x43e1f593f0000001ull, 0x2833e84879b97091ull, 0xb85045b68181585dull, 0x30644e72e131a029ull};
const uint64_t U_BN = 4965661367192848881ull;

uint64_t g_inv = 0;  // -p^-1 mod 2^64
Fq g_r2, g_one;      // R^2 mod p, R mod p

bool geq(const uint64_t* a, const uint64_t* b) {
  for (int i = 3; i >= 0; i--)
    if (a[i] != b[i]) return a[i] > b[i];
  return true;
}

void sub_p(uint64_t* a, const uint64_t* b) {
  uint64_t br = 0;
  for (int i = 0; i < 4; i++) {
    u128 d = (u128)a[i] - b[i] - br;
    a[i] = (uint64_t)d;
    br = (uint64_t)(d >> 64) & 1;
  }
}

Fq fadd(const Fq& a, const Fq& b) {
  Fq r;
  uint64_t c = 0;
  for (int i = 0; i < 4; i++) {
    u128 s = (u128)a.v[i] + b.v[i] + c;
    r.v[i] = (uint64_t)s;
    c = (uint64_t)(s >> 64);
  }
  if (c || geq(r.v, P)) sub_p(r.v, P);
  return r;
}

Fq fsub(const Fq& a, const Fq& b) {
  Fq r;
  uint64_t br = 0;
  for (int i = 0; i < 4; i++) {
    u128 d = (u128)a.v[i] - b.v[i] - br;
    r.v[i] = (uint64_t)d;
    br = (uint64_t)(d >> 64) & 1;
  }
  if (br) {
    uint64_t c = 0;
    for (int i = 0; i < 4; i++) {
      u128 s = (u128)r.v[i] + P[i] + c;
      r.v[i] = (uint64_t)s;
      c = (uint64_t)(s >> 64);
    }
  }
  return r;
}

Fq fneg(const Fq& a) { return fsub(Fq{{0, 0, 0, 0}}, a); }

// CIOS Montgomery product on 4 x 64-bit limbs
Fq fmul(const Fq& a, const Fq& b) {
  uint64_t t[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 4; i++) {
    uint64_t c = 0;
    for (int j = 0; j < 4; j++) {
      u128 s = (u128)a.v[j] * b.v[i] + t[j] + c;
      t[j] = (uint64_t)s;
      c = (uint64_t)(s >> 64);
    }
    u128 s = (u128)t[4] + c;
    t[4] = (uint64_t)s;
    t[5] = (uint64_t)(s >> 64);
    uint64_t m = t[0] * g_inv;
    s = (u128)m * P[0] + t[0];
    c = (uint64_t)(s >> 64);
    for (int j = 1; j < 4; j++) {
      s = (u128)m * P[j] + t[j] + c;
      t[j - 1] = (uint64_t)s;
      c = (uint64_t)(s >> 64);
    }
    s = (u128)t[4] + c;
    t[3] = (uint64_t)s;
    t[4] = t[5] + (uint64_t)(s >> 64);
  }
  Fq r{{t[0], t[1], t[2], t[3]}};
  if (t[4] || geq(r.v, P)) sub_p(r.v, P);
  return r;
}

bool fis_zero(const Fq& a) { return (a.v[0] | a.v[1] | a.v[2] | a.v[3]) == 0; }
bool feq(const Fq& a, const Fq& b) { return memcmp(a.v, b.v, 32) == 0; }

Fq from_u64(uint64_t x) { return fmul(Fq{{x, 0, 0, 0}}, g_r2); }

Fq fpow(Fq a, const uint64_t* e, int limbs) {
  Fq r = g_one;
  for (int i = limbs - 1; i >= 0; i--)
    for (int b = 63; b >= 0; b--) {
      r = fmul(r, r);
      if ((e[i] >> b) & 1) r = fmul(r, a);
    }
  return r;
}

Fq finv(const Fq& a) {
  uint64_t e[4];
  memcpy(e, P, 32);
  e[0] -= 2;
  return fpow(a, e, 4);
}

void init_field() {
  if (g_inv) return;
  uint64_t x = P[0];
  for (int i = 0; i < 6; i++) x *= 2 - P[0] * x;
  g_inv = 0 - x;
  // R mod p and R^2 mod p by doubling 1 (256 and 512 times)
  uint64_t r[4] = {1, 0, 0, 0};
  for (int k = 0; k < 512; k++) {
    uint64_t c = r[3] >> 63;
    for (int i = 3; i > 0; i--) r[i] = (r[i] << 1) | (r[i - 1] >> 63);
    r[0] <<= 1;
    if (c || geq(r, P)) sub_p(r, P);
    if (k == 255) memcpy(g_one.v, r, 32);
  }
  memcpy(g_r2.v, r, 32);
}

// canonical 32 bytes (LE) -> Montgomery; false if not < p
bool load_fq(const uint8_t* b, Fq* out) {
  Fq x;
  for (int i = 0; i < 4; i++) {
    uint64_t w = 0;
    for (int j = 7; j >= 0; j--) w = (w << 8) | b[8 * i + j];
    x.v[i] = w;
  }
  if (geq(x.v, P)) return false;
  *out = fmul(x, g_r2);
  return true;
}

// ------------------------------------------------------------------ tower
struct Fq2 {
  Fq a, b;  // a + b i
};
struct Fq6 {
  Fq2 c0, c1, c2;  // c0 + c1 v + c2 v^2
};
struct Fq12 {
  Fq6 c0, c1;  // c0 + c1 w
};

Fq2 f2(const Fq& a, const Fq& b) { return {a, b}; }
Fq2 f2_zero() { return {Fq{{0, 0, 0, 0}}, Fq{{0, 0, 0, 0}}}; }
Fq2 f2_one() { return {g_one, Fq{{0, 0, 0, 0}}}; }
Fq2 f2_add(const Fq2& x, const Fq2& y) { return {fadd(x.a, y.a), fadd(x.b, y.b)}; }
Fq2 f2_sub(const Fq2& x, const Fq2& y) { return {fsub(x.a, y.a), fsub(x.b, y.b)}; }
Fq2 f2_neg(const Fq2& x) { return {fneg(x.a), fneg(x.b)}; }
Fq2 f2_conj(const Fq2& x) { return {x.a, fneg(x.b)}; }
Fq2 f2_mul(const Fq2& x, const Fq2& y) {
  Fq t0 = fmul(x.a, y.a), t1 = fmul(x.b, y.b);
  Fq t2 = fmul(fadd(x.a, x.b), fadd(y.a, y.b));
  return {fsub(t0, t1), fsub(fsub(t2, t0), t1)};
}
Fq2 f2_scale(const Fq2& x, const Fq& k) { return {fmul(x.a, k), fmul(x.b, k)}; }
bool f2_is_zero(const Fq2& x) { return fis_zero(x.a) && fis_zero(x.b); }
bool f2_eq(const Fq2& x, const Fq2& y) { return feq(x.a, y.a) && feq(x.b, y.b); }
Fq2 f2_inv(const Fq2& x) {
  Fq n = fadd(fmul(x.a, x.a), fmul(x.b, x.b));
  Fq ni = finv(n);
  return {fmul(x.a, ni), fneg(fmul(x.b, ni))};
}
Fq2 f2_pow(Fq2 x, const uint64_t* e, int limbs) {
  Fq2 r = f2_one();
  for (int i = limbs - 1; i >= 0; i--)
    for (int b = 63; b >= 0; b--) {
      r = f2_mul(r, r);
      if ((e[i] >> b) & 1) r = f2_mul(r, x);
    }
  return r;
}

Fq2 g_xi;  // 9 + i
Fq2 mul_xi(const Fq2& x) { return f2_mul(x, g_xi); }

Fq6 f6_zero() { return {f2_zero(), f2_zero(), f2_zero()}; }
Fq6 f6_one() { return {f2_one(), f2_zero(), f2_zero()}; }
Fq6 f6_add(const Fq6& x, const Fq6& y) { return {f2_add(x.c0, y.c0), f2_add(x.c1, y.c1), f2_add(x.c2, y.c2)}; }
Fq6 f6_sub(const Fq6& x, const Fq6& y) { return {f2_sub(x.c0, y.c0), f2_sub(x.c1, y.c1), f2_sub(x.c2, y.c2)}; }
Fq6 f6_neg(const Fq6& x) { return {f2_neg(x.c0), f2_neg(x.c1), f2_neg(x.c2)}; }
// schoolbook with v^3 = xi
Fq6 f6_mul(const Fq6& x, const Fq6& y) {
  Fq2 t0 = f2_mul(x.c0, y.c0), t1 = f2_mul(x.c1, y.c1), t2 = f2_mul(x.c2, y.c2);
  Fq2 c0 = f2_add(t0, mul_xi(f2_add(f2_mul(x.c1, y.c2), f2_mul(x.c2, y.c1))));
  Fq2 c1 = f2_add(f2_add(f2_mul(x.c0, y.c1), f2_mul(x.c1, y.c0)), mul_xi(t2));
  Fq2 c2 = f2_add(f2_add(f2_mul(x.c0, y.c2), f2_mul(x.c2, y.c0)), t1);
  return {c0, c1, c2};
}
Fq6 f6_mul_v(const Fq6& x) { return {mul_xi(x.c2), x.c0, x.c1}; }  // x * v
Fq6 f6_inv(const Fq6& x) {
  // standard: A = c0^2 - xi c1 c2, B = xi c2^2 - c0 c1, C = c1^2 - c0 c2,
  // F = c0 A + xi (c2 B + c1 C), inverse = (A, B, C) / F
  Fq2 A = f2_sub(f2_mul(x.c0, x.c0), mul_xi(f2_mul(x.c1, x.c2)));
  Fq2 B = f2_sub(mul_xi(f2_mul(x.c2, x.c2)), f2_mul(x.c0, x.c1));
  Fq2 C = f2_sub(f2_mul(x.c1, x.c1), f2_mul(x.c0, x.c2));
  Fq2 F = f2_add(f2_mul(x.c0, A), mul_xi(f2_add(f2_mul(x.c2, B), f2_mul(x.c1, C))));
  Fq2 Fi = f2_inv(F);
  return {f2_mul(A, Fi), f2_mul(B, Fi), f2_mul(C, Fi)};
}

Fq12 f12_one() { return {f6_one(), f6_zero()}; }
Fq12 f12_mul(const Fq12& x, const Fq12& y) {
  Fq6 t0 = f6_mul(x.c0, y.c0), t1 = f6_mul(x.c1, y.c1);
  Fq6 c1 = f6_sub(f6_sub(f6_mul(f6_add(x.c0, x.c1), f6_add(y.c0, y.c1)), t0), t1);
  return {f6_add(t0, f6_mul_v(t1)), c1};
}
Fq12 f12_conj(const Fq12& x) { return {x.c0, f6_neg(x.c1)}; }
Fq12 f12_inv(const Fq12& x) {
  // (c0 + c1 w)^-1 = (c0 - c1 w) / (c0^2 - c1^2 v)
  Fq6 d = f6_sub(f6_mul(x.c0, x.c0), f6_mul_v(f6_mul(x.c1, x.c1)));
  Fq6 di = f6_inv(d);
  return {f6_mul(x.c0, di), f6_neg(f6_mul(x.c1, di))};
}
bool f12_is_one(const Fq12& x) {
  Fq12 o = f12_one();
  return memcmp(&x, &o, sizeof(Fq12)) == 0;
}

// ------------------------------------------------------------------ big exponents
typedef std::vector<uint32_t> Big;

Big big_from(const uint64_t* x, int limbs) {
  Big b;
  for (int i = 0; i < limbs; i++) {
    b.push_back((uint32_t)x[i]);
    b.push_back((uint32_t)(x[i] >> 32));
  }
  while (!b.empty() && b.back() == 0) b.pop_back();
  return b;
}
Big big_mul(const Big& a, const Big& b) {
  Big r(a.size() + b.size(), 0);
  for (size_t i = 0; i < a.size(); i++) {
    uint64_t c = 0;
    for (size_t j = 0; j < b.size(); j++) {
      uint64_t s = (uint64_t)a[i] * b[j] + r[i + j] + c;
      r[i + j] = (uint32_t)s;
      c = s >> 32;
    }
    size_t k = i + b.size();
    while (c) {
      uint64_t s = (uint64_t)r[k] + c;
      r[k++] = (uint32_t)s;
      c = s >> 32;
    }
  }
  while (!r.empty() && r.back() == 0) r.pop_back();
  return r;
}
Big big_add_small(Big a, uint32_t x) {
  uint64_t c = x;
  for (size_t i = 0; c && i < a.size(); i++) {
    uint64_t s = (uint64_t)a[i] + c;
    a[i] = (uint32_t)s;
    c = s >> 32;
  }
  if (c) a.push_back((uint32_t)c);
  return a;
}
int big_bits(const Big& a) {
  if (a.empty()) return 0;
  int b = 32 * (int)(a.size() - 1);
  uint32_t t = a.back();
  while (t) {
    b++;
    t >>= 1;
  }
  return b;
}
bool big_bit(const Big& a, int i) { return (a[i / 32] >> (i % 32)) & 1; }
// quotient of a by d (bitwise long division)
Big big_div(const Big& a, const Big& d) {
  int nb = big_bits(a);
  Big q((a.size()) + 1, 0), rem;
  for (int i = nb - 1; i >= 0; i--) {
    // rem = rem * 2 + bit
    uint32_t c = big_bit(a, i) ? 1 : 0;
    for (size_t k = 0; k < rem.size(); k++) {
      uint32_t nc = rem[k] >> 31;
      rem[k] = (rem[k] << 1) | c;
      c = nc;
    }
    if (c) rem.push_back(c);
    // if rem >= d: rem -= d, set bit
    bool ge = rem.size() > d.size();
    if (rem.size() == d.size()) {
      ge = true;
      for (int k = (int)d.size() - 1; k >= 0; k--)
        if (rem[k] != d[k]) {
          ge = rem[k] > d[k];
          break;
        }
    }
    if (ge) {
      int64_t br = 0;
      for (size_t k = 0; k < rem.size(); k++) {
        int64_t s = (int64_t)rem[k] - (k < d.size() ? d[k] : 0) - br;
        br = s < 0;
        rem[k] = (uint32_t)s;
      }
      while (!rem.empty() && rem.back() == 0) rem.pop_back();
      q[i / 32] |= 1u << (i % 32);
    }
  }
  while (!q.empty() && q.back() == 0) q.pop_back();
  return q;
}

Big g_hard;                  // (p^6 + 1) / r
Fq2 g_frob_x, g_frob_y;      // xi^((p-1)/3), xi^((p-1)/2)
Fq2 g_frob2_x, g_frob2_y;    // xi^((p^2-1)/3), xi^((p^2-1)/2)
Fq2 g_b2;                    // 3 / xi
Fq g_b1;                     // 3
bool g_ready = false;

Fq12 f12_pow_big(const Fq12& x, const Big& e) {
  Fq12 r = f12_one();
  for (int i = big_bits(e) - 1; i >= 0; i--) {
    r = f12_mul(r, r);
    if (big_bit(e, i)) r = f12_mul(r, x);
  }
  return r;
}

Fq2 f2_pow_big(const Fq2& x, const Big& e) {
  Fq2 r = f2_one();
  for (int i = big_bits(e) - 1; i >= 0; i--) {
    r = f2_mul(r, r);
    if (big_bit(e, i)) r = f2_mul(r, x);
  }
  return r;
}

void init_all() {
  if (g_ready) return;
  init_field();
  g_xi = f2(from_u64(9), from_u64(1));
  g_b1 = from_u64(3);
  g_b2 = f2_mul(f2(from_u64(3), Fq{{0, 0, 0, 0}}), f2_inv(g_xi));
  Big p = big_from(P, 4), r = big_from(R, 4);
  Big p2 = big_mul(p, p);
  Big p6 = big_mul(big_mul(p2, p2), p2);
  g_hard = big_div(big_add_small(p6, 1), r);
  Big pm1 = p;
  pm1[0] -= 1;  // p is odd: no borrow
  Big p2m1 = p2;
  p2m1[0] -= 1;
  g_frob_x = f2_pow_big(g_xi, big_div(pm1, Big{3}));
  g_frob_y = f2_pow_big(g_xi, big_div(pm1, Big{2}));
  g_frob2_x = f2_pow_big(g_xi, big_div(p2m1, Big{3}));
  g_frob2_y = f2_pow_big(g_xi, big_div(p2m1, Big{2}));
  g_ready = true;
}

// ------------------------------------------------------------------ groups
struct G1 {
  Fq x, y;
  bool inf;
};
struct G2 {
  Fq2 x, y;
  bool inf;
};

bool g1_on_curve(const G1& P1) {
  if (P1.inf) return true;
  return feq(fmul(P1.y, P1.y), fadd(fmul(fmul(P1.x, P1.x), P1.x), g_b1));
}
bool g2_on_curve(const G2& Q) {
  if (Q.inf) return true;
  return f2_eq(f2_mul(Q.y, Q.y), f2_add(f2_mul(f2_mul(Q.x, Q.x), Q.x), g_b2));
}

bool load_g1(const uint8_t* b, G1* out) {
  static const uint8_t zero[64] = {0};
  if (memcmp(b, zero, 64) == 0) {
    out->inf = true;
    return true;
  }
  out->inf = false;
  return load_fq(b, &out->x) && load_fq(b + 32, &out->y);
}
bool load_g2(const uint8_t* b, G2* out) {
  static const uint8_t zero[128] = {0};
  if (memcmp(b, zero, 128) == 0) {
    out->inf = true;
    return true;
  }
  out->inf = false;
  return load_fq(b, &out->x.a) && load_fq(b + 32, &out->x.b) && load_fq(b + 64, &out->y.a) &&
         load_fq(b + 96, &out->y.b);
}

// Jacobian G1 for the public-input sum
struct G1J {
  Fq X, Y, Z;  // Z = 0: infinity
};
G1J j_inf() { return {g_one, g_one, Fq{{0, 0, 0, 0}}}; }
G1J j_dbl(const G1J& p) {
  if (fis_zero(p.Z) || fis_zero(p.Y)) return j_inf();
  Fq A = fmul(p.X, p.X), B = fmul(p.Y, p.Y), C = fmul(B, B);
  Fq t = fadd(p.X, B);
  Fq D = fsub(fsub(fmul(t, t), A), C);
  D = fadd(D, D);
  Fq E = fadd(fadd(A, A), A);
  Fq F = fmul(E, E);
  Fq X3 = fsub(F, fadd(D, D));
  Fq C8 = fadd(C, C);
  C8 = fadd(C8, C8);
  C8 = fadd(C8, C8);
  Fq Y3 = fsub(fmul(E, fsub(D, X3)), C8);
  Fq Z3 = fmul(p.Y, p.Z);
  return {X3, Y3, fadd(Z3, Z3)};
}
G1J j_add_affine(const G1J& p, const G1& q) {
  if (q.inf) return p;
  if (fis_zero(p.Z)) return {q.x, q.y, g_one};
  Fq Z1Z1 = fmul(p.Z, p.Z);
  Fq U2 = fmul(q.x, Z1Z1), S2 = fmul(fmul(q.y, p.Z), Z1Z1);
  Fq H = fsub(U2, p.X), rr = fsub(S2, p.Y);
  if (fis_zero(H)) {
    if (fis_zero(rr)) return j_dbl({q.x, q.y, g_one});
    return j_inf();
  }
  Fq HH = fmul(H, H), HHH = fmul(H, HH), V = fmul(p.X, HH);
  Fq X3 = fsub(fsub(fmul(rr, rr), HHH), fadd(V, V));
  Fq Y3 = fsub(fmul(rr, fsub(V, X3)), fmul(p.Y, HHH));
  return {X3, Y3, fmul(p.Z, H)};
}
G1 j_to_affine(const G1J& p) {
  if (fis_zero(p.Z)) return {g_one, g_one, true};
  Fq zi = finv(p.Z), zi2 = fmul(zi, zi);
  return {fmul(p.X, zi2), fmul(fmul(p.Y, zi2), zi), false};
}
G1 g1_neg(const G1& p) { return {p.x, fneg(p.y), p.inf}; }

// sum_k s_k P_k for small signed scalars (|s| < 2^31): buckets by byte, four 8-bit windows
G1 small_msm(const std::vector<G1>& pts, const std::vector<int64_t>& sc) {
  G1J total = j_inf();
  for (int w = 3; w >= 0; w--) {
    for (int i = 0; i < 8; i++) total = j_dbl(total);
    G1J buckets[256];
    for (auto& b : buckets) b = j_inf();
    for (size_t k = 0; k < pts.size(); k++) {
      int64_t s = sc[k];
      uint64_t m = (uint64_t)(s < 0 ? -s : s);
      uint32_t d = (m >> (8 * w)) & 255u;
      if (!d) continue;
      buckets[d] = j_add_affine(buckets[d], s < 0 ? g1_neg(pts[k]) : pts[k]);
    }
    // sum_d d B_d by running sums
    G1J run = j_inf(), acc = j_inf();
    for (int d = 255; d >= 1; d--) {
      if (!fis_zero(buckets[d].Z)) {
        G1 ba = j_to_affine(buckets[d]);
        run = j_add_affine(run, ba);
      }
      if (!fis_zero(run.Z)) acc = j_add_affine(acc, j_to_affine(run));
    }
    if (!fis_zero(acc.Z)) total = j_add_affine(total, j_to_affine(acc));
  }
  return j_to_affine(total);
}

// [r] Q == O on the twist (affine double-and-add over the bits of r)
G2 g2_add(const G2& p, const G2& q) {
  if (p.inf) return q;
  if (q.inf) return p;
  Fq2 lam;
  if (f2_eq(p.x, q.x)) {
    if (f2_is_zero(f2_add(p.y, q.y))) return {f2_zero(), f2_zero(), true};
    Fq2 x2 = f2_mul(p.x, p.x);
    lam = f2_mul(f2_add(f2_add(x2, x2), x2), f2_inv(f2_add(p.y, p.y)));
  } else {
    lam = f2_mul(f2_sub(q.y, p.y), f2_inv(f2_sub(q.x, p.x)));
  }
  Fq2 x3 = f2_sub(f2_sub(f2_mul(lam, lam), p.x), q.x);
  Fq2 y3 = f2_sub(f2_mul(lam, f2_sub(p.x, x3)), p.y);
  return {x3, y3, false};
}
bool g2_in_subgroup(const G2& Q) {
  if (Q.inf) return true;
  G2 acc{f2_zero(), f2_zero(), true};
  for (int i = 3; i >= 0; i--)
    for (int b = 63; b >= 0; b--) {
      acc = g2_add(acc, acc);
      if ((R[i] >> b) & 1) acc = g2_add(acc, Q);
    }
  return acc.inf;
}

// ------------------------------------------------------------------ Miller loop
// line through T (and Q, or the tangent at T) on the twist, evaluated at P
Fq12 line_eval(const Fq2& lam, const Fq2& xT, const Fq2& yT, const G1& P1) {
  Fq12 l;
  l.c0 = f6_zero();
  l.c0.c0 = f2(P1.y, Fq{{0, 0, 0, 0}});
  l.c1 = f6_zero();
  l.c1.c0 = f2_neg(f2_scale(lam, P1.x));
  l.c1.c1 = f2_sub(f2_mul(lam, xT), yT);
  return l;
}

// f = f * line(T, Q) and T = T + Q (Q may equal T: tangent); vertical lines are dropped
// (they lie in a proper subfield and vanish in the final exponentiation)
void step(Fq12& f, G2& T, const G2& Q, const G1& P1) {
  if (T.inf || Q.inf) {
    T = g2_add(T, Q);
    return;
  }
  Fq2 lam;
  if (f2_eq(T.x, Q.x)) {
    if (!f2_eq(T.y, Q.y)) {  // vertical
      T = {f2_zero(), f2_zero(), true};
      return;
    }
    Fq2 x2 = f2_mul(T.x, T.x);
    lam = f2_mul(f2_add(f2_add(x2, x2), x2), f2_inv(f2_add(T.y, T.y)));
  } else {
    lam = f2_mul(f2_sub(Q.y, T.y), f2_inv(f2_sub(Q.x, T.x)));
  }
  f = f12_mul(f, line_eval(lam, T.x, T.y, P1));
  Fq2 x3 = f2_sub(f2_sub(f2_mul(lam, lam), T.x), Q.x);
  Fq2 y3 = f2_sub(f2_mul(lam, f2_sub(T.x, x3)), T.y);
  T = {x3, y3, false};
}

Fq12 miller(const G1& P1, const G2& Q) {
  if (P1.inf || Q.inf) return f12_one();
  const uint64_t loop = 6 * U_BN + 2;  // fits in 65 bits? 6u + 2 < 2^65: handle as u128
  u128 L = (u128)6 * U_BN + 2;
  (void)loop;
  int top = 127;
  while (!((L >> top) & 1)) top--;
  Fq12 f = f12_one();
  G2 T = Q;
  for (int i = top - 1; i >= 0; i--) {
    f = f12_mul(f, f);
    step(f, T, T, P1);
    if ((L >> i) & 1) step(f, T, Q, P1);
  }
  G2 Q1{f2_mul(f2_conj(Q.x), g_frob_x), f2_mul(f2_conj(Q.y), g_frob_y), false};
  G2 Q2{f2_mul(Q.x, g_frob2_x), f2_mul(Q.y, g_frob2_y), false};
  G2 nQ2{Q2.x, f2_neg(Q2.y), false};
  step(f, T, Q1, P1);
  step(f, T, nQ2, P1);
  return f;
}

Fq12 final_exp(const Fq12& f) {
  Fq12 t = f12_mul(f12_conj(f), f12_inv(f));  // f^(p^6 - 1)
  return f12_pow_big(t, g_hard);
}

}  // namespace

struct zkvc_vk;

namespace zkvc {
// vk accessors (defined with the vk struct in the CUDA translation unit)
int vk_get(const zkvc_vk* vk, int* a, int* n, int* b, const uint8_t** alpha1, const uint8_t** beta2,
           const uint8_t** gamma2, const uint8_t** delta2, const uint8_t** ic, size_t* n_ic);

int verify_impl(const zkvc_vk* vk, const int8_t* X, const int32_t* Y, const uint8_t* proof, int* ok) {
  init_all();
  int a = 0, n = 0, b = 0;
  const uint8_t *alpha1, *beta2, *gamma2, *delta2, *ic;
  size_t n_ic = 0;
  int rc = vk_get(vk, &a, &n, &b, &alpha1, &beta2, &gamma2, &delta2, &ic, &n_ic);
  if (rc != ZKVC_OK) return rc;
  *ok = 0;
  G1 A, C, al;
  G2 B, be, ga, de;
  if (!load_g1(proof, &A) || !load_g2(proof + 64, &B) || !load_g1(proof + 192, &C)) return ZKVC_OK;
  if (!g1_on_curve(A) || !g1_on_curve(C) || !g2_on_curve(B) || !g2_in_subgroup(B)) return ZKVC_OK;
  if (!load_g1(alpha1, &al) || !load_g2(beta2, &be) || !load_g2(gamma2, &ga) || !load_g2(delta2, &de)) {
    set_error("verify: corrupt verifying key");
    return ZKVC_EIO;
  }
  // IC(x) = IC_0 + sum_v x_v IC_v over the public inputs X (row-major) then Y (row-major);
  // a key without public inputs (X and Y private) holds IC_0 alone
  size_t l = size_t(a) * n + size_t(a) * b;
  if (n_ic == 1) l = 0;
  if (n_ic != l + 1) {
    set_error("verify: verifying key has %zu IC points for %zu public inputs", n_ic, l);
    return ZKVC_EIO;
  }
  std::vector<G1> pts(l);
  std::vector<int64_t> sc(l);
  for (size_t v = 0; v < l; v++) {
    if (!load_g1(ic + 64 * (v + 1), &pts[v])) {
      set_error("verify: corrupt IC point");
      return ZKVC_EIO;
    }
    sc[v] = v < size_t(a) * n ? (int64_t)X[v] : (int64_t)Y[v - size_t(a) * n];
  }
  G1 ic0;
  load_g1(ic, &ic0);
  G1 sum = small_msm(pts, sc);
  G1J acc = j_add_affine(j_add_affine(j_inf(), ic0), sum);
  G1 icx = j_to_affine(acc);
  Fq12 f = miller(g1_neg(A), B);
  f = f12_mul(f, miller(al, be));
  f = f12_mul(f, miller(icx, ga));
  f = f12_mul(f, miller(C, de));
  *ok = f12_is_one(final_exp(f)) ? 1 : 0;
  return ZKVC_OK;
}

}  // namespace zkvc
