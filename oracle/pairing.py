"""Optimal-ate pairing on BN254, textbook form.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Groth16 verification (zkVC Sec. II: Gen / Prove / Verify; the paper's groth16 backend
checks proofs with a pairing equation) needs a bilinear, non-degenerate pairing
e: G1 x G2 -> GT.  This module computes it as plainly as possible:

* Fp12 is represented as Fp[w]/(w^12 - 18 w^6 + 82): with w^6 = xi = 9 + i this is the
  same field as Fp2[w]/(w^6 - xi), since i = w^6 - 9 and i^2 = -1.
* A G2 point (x, y) on the twist is mapped into E(Fp12) by (x w^2, y w^3).
* The Miller loop runs over the bits of 6u + 2 with affine points over Fp12 and the
  chord/tangent line functions evaluated at P; vertical lines are dropped because they
  lie in a proper subfield and vanish under the final exponentiation.
* Two extra lines with pi(Q) and -pi^2(Q) (Frobenius) complete the optimal-ate loop.
* The final exponentiation is plain square-and-multiply by (p^12 - 1)/r.

Pins (tests/test_oracle_pairing.py): bilinearity in both arguments, non-degeneracy,
e^r = 1, and e(P, Q) = e(Q-side twist consistency) through random multiples.
"""
from .bn254 import P, R, ATE_LOOP, g1_neg

DEG = 12
# w^12 = 18 w^6 - 82
_MOD_W6 = 18
_MOD_W0 = -82
FINAL_EXP = (P**12 - 1) // R


def f12(coeffs):
    c = [0] * DEG
    for k, v in enumerate(coeffs):
        c[k] = v % P
    return tuple(c)


F12_ONE = f12([1])
F12_ZERO = f12([])


def f12_add(a, b):
    return tuple((x + y) % P for x, y in zip(a, b))


def f12_sub(a, b):
    return tuple((x - y) % P for x, y in zip(a, b))


def f12_neg(a):
    return tuple((-x) % P for x in a)


def f12_mul(a, b):
    prod = [0] * (2 * DEG - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                prod[i + j] += x * y
    # reduce: w^d = w^(d-12) (18 w^6 - 82) for d >= 12, from the top down
    for d in range(2 * DEG - 2, DEG - 1, -1):
        c = prod[d]
        if c:
            prod[d - 6] += _MOD_W6 * c
            prod[d - 12] += _MOD_W0 * c
    return tuple(v % P for v in prod[:DEG])


def f12_scale(a, k):
    return tuple(x * k % P for x in a)


def _poly_deg(p):
    d = len(p) - 1
    while d >= 0 and p[d] % P == 0:
        d -= 1
    return d


def _poly_divmod(num, den):
    num = [v % P for v in num]
    dd = _poly_deg(den)
    inv_lead = pow(den[dd], -1, P)
    q = [0] * max(1, len(num) - dd)
    for k in range(len(num) - 1, dd - 1, -1):
        c = num[k] * inv_lead % P
        if c:
            q[k - dd] = c
            for j in range(dd + 1):
                num[k - dd + j] = (num[k - dd + j] - c * den[j]) % P
    return q, num[:dd] if dd > 0 else [0]


def f12_inv(a):
    """Inverse by the extended Euclidean algorithm on polynomials over Fp."""
    modulus = [82, 0, 0, 0, 0, 0, (-18) % P, 0, 0, 0, 0, 0, 1]
    r0, r1 = modulus, list(a)
    s0, s1 = [0], [1]
    if _poly_deg(r1) < 0:
        raise ZeroDivisionError("inverse of 0 in Fp12")
    while _poly_deg(r1) > 0:
        q, rem = _poly_divmod(r0, r1[:_poly_deg(r1) + 1])
        # s_{k+1} = s_{k-1} - q s_k
        prod = [0] * (len(q) + len(s1) - 1)
        for i, x in enumerate(q):
            for j, y in enumerate(s1):
                prod[i + j] += x * y
        n = max(len(s0), len(prod))
        s2 = [((s0[i] if i < len(s0) else 0) - (prod[i] if i < len(prod) else 0)) % P
              for i in range(n)]
        r0, r1, s0, s1 = r1, rem, s1, s2
    c = pow(r1[0], -1, P)
    # reduce s1 modulo the field polynomial, then scale
    _, red = _poly_divmod(s1 + [0] * max(0, DEG + 1 - len(s1)), modulus)
    red = list(red) + [0] * (DEG - len(red))
    return tuple(v * c % P for v in red[:DEG])


def f12_pow(a, e):
    out = F12_ONE
    base = a
    for bit in bin(e)[2:]:
        out = f12_mul(out, out)
        if bit == "1":
            out = f12_mul(out, a)
    return out


def fp2_to_f12(z):
    """a + b i  ->  (a - 9 b) + b w^6, using i = w^6 - 9."""
    a, b = z
    c = [0] * DEG
    c[0] = (a - 9 * b) % P
    c[6] = b % P
    return tuple(c)


def _w_pow(k):
    c = [0] * DEG
    c[k] = 1
    return tuple(c)


_W2 = _w_pow(2)
_W3 = _w_pow(3)


def untwist(Q):
    """E'(Fp2) -> E(Fp12): (x, y) -> (x w^2, y w^3)."""
    if Q is None:
        return None
    x, y = Q
    return (f12_mul(fp2_to_f12(x), _W2), f12_mul(fp2_to_f12(y), _W3))


def embed_g1(Pt):
    if Pt is None:
        return None
    return (f12([Pt[0]]), f12([Pt[1]]))


def e12_add(A, B):
    """Affine addition on y^2 = x^3 + 3 with coordinates in Fp12."""
    if A is None:
        return B
    if B is None:
        return A
    x1, y1 = A
    x2, y2 = B
    if x1 == x2:
        if f12_add(y1, y2) == F12_ZERO:
            return None
        lam = f12_mul(f12_scale(f12_mul(x1, x1), 3), f12_inv(f12_scale(y1, 2)))
    else:
        lam = f12_mul(f12_sub(y2, y1), f12_inv(f12_sub(x2, x1)))
    x3 = f12_sub(f12_sub(f12_mul(lam, lam), x1), x2)
    y3 = f12_sub(f12_mul(lam, f12_sub(x1, x3)), y1)
    return (x3, y3)


def line(T, Q, Pt):
    """Value at Pt of the line through T and Q (the tangent when T = Q)."""
    x1, y1 = T
    x2, y2 = Q
    xp, yp = Pt
    if x1 != x2:
        lam = f12_mul(f12_sub(y2, y1), f12_inv(f12_sub(x2, x1)))
    elif y1 == y2:
        lam = f12_mul(f12_scale(f12_mul(x1, x1), 3), f12_inv(f12_scale(y1, 2)))
    else:
        return f12_sub(xp, x1)                 # vertical line
    return f12_sub(f12_mul(lam, f12_sub(xp, x1)), f12_sub(yp, y1))


def frobenius_point(T):
    return (f12_pow(T[0], P), f12_pow(T[1], P))


def miller_loop(Pt, Q):
    """f_{6u+2,Q}(P) times the two Frobenius lines of the optimal-ate pairing."""
    if Pt is None or Q is None:
        return F12_ONE
    Pe = embed_g1(Pt)
    Qe = untwist(Q)
    T = Qe
    f = F12_ONE
    for bit in bin(ATE_LOOP)[3:]:
        f = f12_mul(f12_mul(f, f), line(T, T, Pe))
        T = e12_add(T, T)
        if bit == "1":
            f = f12_mul(f, line(T, Qe, Pe))
            T = e12_add(T, Qe)
    Q1 = frobenius_point(Qe)
    Q2 = frobenius_point(Q1)
    nQ2 = (Q2[0], f12_neg(Q2[1]))
    f = f12_mul(f, line(T, Q1, Pe))
    T = e12_add(T, Q1)
    f = f12_mul(f, line(T, nQ2, Pe))
    return f


def final_exponentiation(f):
    return f12_pow(f, FINAL_EXP)


def pairing(Pt, Q):
    """e(P, Q) for P in G1 (affine over Fp) and Q in G2 (affine over Fp2)."""
    return final_exponentiation(miller_loop(Pt, Q))


def pairing_product_is_one(pairs):
    """True iff prod_k e(P_k, Q_k) = 1 (one shared final exponentiation)."""
    f = F12_ONE
    for Pt, Q in pairs:
        f = f12_mul(f, miller_loop(Pt, Q))
    return final_exponentiation(f) == F12_ONE


__all__ = ["pairing", "pairing_product_is_one", "miller_loop", "final_exponentiation",
           "f12_mul", "f12_pow", "f12_inv", "F12_ONE", "g1_neg"]
