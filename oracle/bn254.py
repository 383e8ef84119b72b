"""BN254 ("alt_bn128") parameters, fields and groups, written out with Python integers.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper runs Groth16 through libsnark (Sec. IV, implementation details) without
naming the curve; libsnark's default pairing curve is BN254 and the workload fixes
BN254, so this module restates that curve from its defining parameter u.

Pins (tests/test_oracle_bn254.py): p and r prime, r = p + 1 - t with t = 6u^2 + 1,
p = 3 mod 4, the generators on their curves with [r]G = O, xi = 9 + i neither a square
nor a cube in Fp2, Jacobian arithmetic against affine arithmetic and brute force.
"""

# ---------------------------------------------------------------- parameters
U = 4965661367192848881                      # BN parameter u
P = 36 * U**4 + 36 * U**3 + 24 * U**2 + 6 * U + 1   # base field modulus p
R = 36 * U**4 + 36 * U**3 + 18 * U**2 + 6 * U + 1   # group order r (scalar field Fr)
TRACE = 6 * U**2 + 1                         # Frobenius trace t, #E(Fp) = p + 1 - t
B1 = 3                                       # G1: y^2 = x^3 + 3 over Fp
XI = (9, 1)                                  # xi = 9 + i, Fp6 = Fp2[v]/(v^3 - xi)
ATE_LOOP = 6 * U + 2                         # optimal-ate loop parameter

# Fr two-adicity and the NTT generator (see tests for the pins).
FR_GEN = 5                                   # quadratic non-residue of Fr, used as
                                             # root source and as the coset shift g
FR_TWO_ADICITY = 28


def is_probable_prime(n, rounds=40):
    """Miller-Rabin with fixed small-prime bases plus deterministic pseudo-random ones."""
    if n < 2:
        return False
    small = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 71]
    for q in small:
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    bases = small[:]
    x = 0x1234567
    while len(bases) < rounds:
        x = (x * 6364136223846793005 + 1442695040888963407) % (1 << 64)
        bases.append(2 + x % (n - 3))
    for a in bases:
        y = pow(a, d, n)
        if y in (1, n - 1):
            continue
        for _ in range(s - 1):
            y = y * y % n
            if y == n - 1:
                break
        else:
            return False
    return True


# ---------------------------------------------------------------- Fr helpers
def fr_inv(a):
    a %= R
    if a == 0:
        raise ZeroDivisionError("inverse of 0 in Fr")
    return pow(a, -1, R)


def fr_from_int(v):
    """Map a signed integer to Fr: v >= 0 -> v, v < 0 -> r - |v| (workload convention)."""
    return v % R


def fr_root_of_unity(n):
    """Primitive n-th root of unity omega_n = g^((r-1)/2^28) ^ (2^28/n), n a power of 2."""
    assert n & (n - 1) == 0 and 1 <= n <= (1 << FR_TWO_ADICITY)
    w28 = pow(FR_GEN, (R - 1) >> FR_TWO_ADICITY, R)
    return pow(w28, (1 << FR_TWO_ADICITY) // n, R)


# ---------------------------------------------------------------- Fp2 = Fp[i]/(i^2+1)
def f2_add(a, b):
    return ((a[0] + b[0]) % P, (a[1] + b[1]) % P)


def f2_sub(a, b):
    return ((a[0] - b[0]) % P, (a[1] - b[1]) % P)


def f2_neg(a):
    return ((-a[0]) % P, (-a[1]) % P)


def f2_mul(a, b):
    # (a0 + a1 i)(b0 + b1 i) = (a0 b0 - a1 b1) + (a0 b1 + a1 b0) i
    return ((a[0] * b[0] - a[1] * b[1]) % P, (a[0] * b[1] + a[1] * b[0]) % P)


def f2_scale(a, k):
    return (a[0] * k % P, a[1] * k % P)


def f2_inv(a):
    # 1/(a0 + a1 i) = (a0 - a1 i)/(a0^2 + a1^2)
    n = (a[0] * a[0] + a[1] * a[1]) % P
    ni = pow(n, -1, P)
    return (a[0] * ni % P, (-a[1]) * ni % P)


def f2_pow(a, e):
    out = (1, 0)
    base = a
    while e:
        if e & 1:
            out = f2_mul(out, base)
        base = f2_mul(base, base)
        e >>= 1
    return out


F2_ZERO = (0, 0)
F2_ONE = (1, 0)

# G2 twist coefficient b' = 3 / xi  (D-type sextic twist y^2 = x^3 + 3/xi)
B2 = f2_mul((3, 0), f2_inv(XI))


# ---------------------------------------------------------------- G1 (affine, None = O)
G1_GEN = (1, 2)


def g1_on_curve(Pt):
    if Pt is None:
        return True
    x, y = Pt
    return (y * y - x * x * x - B1) % P == 0


def g1_neg(Pt):
    if Pt is None:
        return None
    return (Pt[0], (-Pt[1]) % P)


def g1_add(P1, P2):
    """Textbook affine chord-and-tangent addition on y^2 = x^3 + 3."""
    if P1 is None:
        return P2
    if P2 is None:
        return P1
    x1, y1 = P1
    x2, y2 = P2
    if x1 == x2:
        if (y1 + y2) % P == 0:
            return None
        lam = 3 * x1 * x1 * pow(2 * y1, -1, P) % P
    else:
        lam = (y2 - y1) * pow(x2 - x1, -1, P) % P
    x3 = (lam * lam - x1 - x2) % P
    y3 = (lam * (x1 - x3) - y1) % P
    return (x3, y3)


# Jacobian coordinates (X, Y, Z): x = X/Z^2, y = Y/Z^3; Z = 0 is O.  Used only to make the
# many scalar multiplications of the oracle affordable; pinned against g1_add.
def _jac_dbl(X, Y, Z):
    if Z == 0 or Y == 0:
        return (1, 1, 0)
    A = X * X % P
    Bv = Y * Y % P
    C = Bv * Bv % P
    D = 2 * ((X + Bv) * (X + Bv) - A - C) % P
    E = 3 * A % P
    F = E * E % P
    X3 = (F - 2 * D) % P
    Y3 = (E * (D - X3) - 8 * C) % P
    Z3 = 2 * Y * Z % P
    return (X3, Y3, Z3)


def _jac_add_affine(X1, Y1, Z1, x2, y2):
    if Z1 == 0:
        return (x2, y2, 1)
    Z1Z1 = Z1 * Z1 % P
    U2 = x2 * Z1Z1 % P
    S2 = y2 * Z1 * Z1Z1 % P
    H = (U2 - X1) % P
    rr = (S2 - Y1) % P
    if H == 0:
        if rr == 0:
            return _jac_dbl(X1, Y1, Z1)
        return (1, 1, 0)
    HH = H * H % P
    HHH = H * HH % P
    V = X1 * HH % P
    X3 = (rr * rr - HHH - 2 * V) % P
    Y3 = (rr * (V - X3) - Y1 * HHH) % P
    Z3 = Z1 * H % P
    return (X3, Y3, Z3)


def _jac_to_affine(X, Y, Z):
    if Z == 0:
        return None
    zi = pow(Z, -1, P)
    zi2 = zi * zi % P
    return (X * zi2 % P, Y * zi2 * zi % P)


def g1_mul(Pt, k):
    """[k]P by MSB-first double-and-add on the canonical scalar k mod r.

    Shortcut: for k > (r-1)/2 compute -[r-k]P, valid because [r]P = O on G1 (pinned).
    """
    k %= R
    if Pt is None or k == 0:
        return None
    if k > (R - 1) // 2:
        return g1_neg(g1_mul(Pt, R - k))
    x, y = Pt
    X, Y, Z = (1, 1, 0)
    for bit in bin(k)[2:]:
        X, Y, Z = _jac_dbl(X, Y, Z)
        if bit == "1":
            X, Y, Z = _jac_add_affine(X, Y, Z, x, y)
    return _jac_to_affine(X, Y, Z)


def g1_mul_noshortcut(Pt, k):
    """[k]P for any non-negative integer k (no reduction mod r); used by the [r]G = O pin."""
    if Pt is None or k == 0:
        return None
    x, y = Pt
    X, Y, Z = (1, 1, 0)
    for bit in bin(k)[2:]:
        X, Y, Z = _jac_dbl(X, Y, Z)
        if bit == "1":
            X, Y, Z = _jac_add_affine(X, Y, Z, x, y)
    return _jac_to_affine(X, Y, Z)


def g1_msm(points, scalars):
    """Naive multi-scalar multiplication: the sum of [s_i]P_i, one scalar mult per term."""
    acc = None
    for Pt, s in zip(points, scalars):
        if s % R:
            acc = g1_add(acc, g1_mul(Pt, s))
    return acc


# ---------------------------------------------------------------- G2 over Fp2 (affine)
# Generator of the order-r subgroup of E'(Fp2) as published with EIP-197 (x = x0 + x1 i,
# y = y0 + y1 i); pinned by the on-curve and [r]Q = O tests.
G2_GEN = (
    (10857046999023057135944570762232829481370756359578518086990519993285655852781,
     11559732032986387107991004021392285783925812861821192530917403151452391805634),
    (8495653923123431417604973247489272438418190587263600148770280649306958101930,
     4082367875863433681332203403145435568316851327593401208105741076214120093531),
)


def g2_on_curve(Q):
    if Q is None:
        return True
    x, y = Q
    lhs = f2_mul(y, y)
    rhs = f2_add(f2_mul(f2_mul(x, x), x), B2)
    return lhs == rhs


def g2_neg(Q):
    if Q is None:
        return None
    return (Q[0], f2_neg(Q[1]))


def g2_add(Q1, Q2):
    """Textbook affine addition on the twist y^2 = x^3 + 3/xi over Fp2."""
    if Q1 is None:
        return Q2
    if Q2 is None:
        return Q1
    x1, y1 = Q1
    x2, y2 = Q2
    if x1 == x2:
        if f2_add(y1, y2) == F2_ZERO:
            return None
        lam = f2_mul(f2_scale(f2_mul(x1, x1), 3), f2_inv(f2_scale(y1, 2)))
    else:
        lam = f2_mul(f2_sub(y2, y1), f2_inv(f2_sub(x2, x1)))
    x3 = f2_sub(f2_sub(f2_mul(lam, lam), x1), x2)
    y3 = f2_sub(f2_mul(lam, f2_sub(x1, x3)), y1)
    return (x3, y3)


def _g2_jac_dbl(X, Y, Z):
    if Z == F2_ZERO or Y == F2_ZERO:
        return (F2_ONE, F2_ONE, F2_ZERO)
    A = f2_mul(X, X)
    Bv = f2_mul(Y, Y)
    C = f2_mul(Bv, Bv)
    t = f2_add(X, Bv)
    D = f2_scale(f2_sub(f2_sub(f2_mul(t, t), A), C), 2)
    E = f2_scale(A, 3)
    F = f2_mul(E, E)
    X3 = f2_sub(F, f2_scale(D, 2))
    Y3 = f2_sub(f2_mul(E, f2_sub(D, X3)), f2_scale(C, 8))
    Z3 = f2_scale(f2_mul(Y, Z), 2)
    return (X3, Y3, Z3)


def _g2_jac_add_affine(X1, Y1, Z1, x2, y2):
    if Z1 == F2_ZERO:
        return (x2, y2, F2_ONE)
    Z1Z1 = f2_mul(Z1, Z1)
    U2 = f2_mul(x2, Z1Z1)
    S2 = f2_mul(f2_mul(y2, Z1), Z1Z1)
    H = f2_sub(U2, X1)
    rr = f2_sub(S2, Y1)
    if H == F2_ZERO:
        if rr == F2_ZERO:
            return _g2_jac_dbl(X1, Y1, Z1)
        return (F2_ONE, F2_ONE, F2_ZERO)
    HH = f2_mul(H, H)
    HHH = f2_mul(H, HH)
    V = f2_mul(X1, HH)
    X3 = f2_sub(f2_sub(f2_mul(rr, rr), HHH), f2_scale(V, 2))
    Y3 = f2_sub(f2_mul(rr, f2_sub(V, X3)), f2_mul(Y1, HHH))
    Z3 = f2_mul(Z1, H)
    return (X3, Y3, Z3)


def _g2_jac_to_affine(X, Y, Z):
    if Z == F2_ZERO:
        return None
    zi = f2_inv(Z)
    zi2 = f2_mul(zi, zi)
    return (f2_mul(X, zi2), f2_mul(f2_mul(Y, zi2), zi))


def g2_mul_noshortcut(Q, k):
    if Q is None or k == 0:
        return None
    x, y = Q
    X, Y, Z = (F2_ONE, F2_ONE, F2_ZERO)
    for bit in bin(k)[2:]:
        X, Y, Z = _g2_jac_dbl(X, Y, Z)
        if bit == "1":
            X, Y, Z = _g2_jac_add_affine(X, Y, Z, x, y)
    return _g2_jac_to_affine(X, Y, Z)


def g2_mul(Q, k):
    """[k]Q, double-and-add on k mod r with the -[r-k]Q shortcut ([r]Q = O is pinned)."""
    k %= R
    if Q is None or k == 0:
        return None
    if k > (R - 1) // 2:
        return g2_neg(g2_mul_noshortcut(Q, R - k))
    return g2_mul_noshortcut(Q, k)


def g2_msm(points, scalars):
    acc = None
    for Q, s in zip(points, scalars):
        if s % R:
            acc = g2_add(acc, g2_mul(Q, s))
    return acc


# ---------------------------------------------------------------- serialisation
def fe_bytes(v):
    """Canonical (non-Montgomery) 32-byte little-endian encoding of a field element."""
    return int(v).to_bytes(32, "little")


def g1_bytes(Pt):
    """Affine G1 point: x || y (64 bytes); the point at infinity is 64 zero bytes."""
    if Pt is None:
        return bytes(64)
    return fe_bytes(Pt[0]) + fe_bytes(Pt[1])


def g2_bytes(Q):
    """Affine G2 point: x.c0 || x.c1 || y.c0 || y.c1 (128 bytes); infinity is all zero."""
    if Q is None:
        return bytes(128)
    return fe_bytes(Q[0][0]) + fe_bytes(Q[0][1]) + fe_bytes(Q[1][0]) + fe_bytes(Q[1][1])


def g1_from_bytes(bs):
    assert len(bs) == 64
    if bs == bytes(64):
        return None
    return (int.from_bytes(bs[:32], "little"), int.from_bytes(bs[32:], "little"))


def g2_from_bytes(bs):
    assert len(bs) == 128
    if bs == bytes(128):
        return None
    v = [int.from_bytes(bs[32 * i:32 * i + 32], "little") for i in range(4)]
    return ((v[0], v[1]), (v[2], v[3]))
