"""Design constants and bounds of two integer algorithms of the CUDA field code, checked
on the CPU with Python integers (no GPU; the GPU parity tests compare the kernels
themselves with the oracle):

* the binary-GCD inversion of field.cuh (Pornin, "Optimized Binary GCD for Modular
  Inversion", 2020): 17 rounds of 30 steps on 62-bit stand-ins of (a, b) reach a = 0,
  b = 1 for both BN254 moduli, every transition matrix entry stays within 2^30 in
  magnitude (32-bit signed factors), every intermediate of the exact update fits the
  288-bit two's complement accumulators, and the Montgomery-style division of (u, v) by
  2^30 leaves v = y^-1 with no final correction;
* the limb-sliced CIOS product of sliced.cuh (eight lanes, one 32-bit limb each): every
  per-lane intermediate fits 64 bits, position 0 becomes zero in each row, the result is
  below 2p after the rows, and the carry-lookahead identity carries = ((G | P) + G) xor P
  reproduces ripple-carry addition for every generate/propagate pattern."""
import itertools
import random

import pytest

from oracle import bn254 as bn

K = 30          # binary-GCD steps per round
ROUNDS = 17     # rounds run by the device code
M32 = (1 << 32) - 1


def _bgcd(y, m, rounds=ROUNDS):
    a, b, u, v = y, m, 1, 0
    minv = (-pow(m, -1, 1 << K)) % (1 << K)
    for _ in range(rounds):
        n = max(a.bit_length(), b.bit_length(), 2 * K + 2)
        ab = (a & ((1 << K) - 1)) | ((a >> (n - K - 2)) << K)
        bb = (b & ((1 << K) - 1)) | ((b >> (n - K - 2)) << K)
        assert ab < 1 << 64 and bb < 1 << 64
        f0, g0, f1, g1 = 1, 0, 0, 1
        for _ in range(K):
            if ab & 1:
                if ab < bb:
                    ab, bb, f0, g0, f1, g1 = bb, ab, f1, g1, f0, g0
                ab = (ab - bb) >> 1
                f0, g0 = f0 - f1, g0 - g1
            else:
                ab >>= 1
            f1, g1 = 2 * f1, 2 * g1
        assert max(abs(f0), abs(g0), abs(f1), abs(g1)) <= 1 << K
        ta, tb = a * f0 + b * g0, a * f1 + b * g1
        assert ta % (1 << K) == 0 and tb % (1 << K) == 0
        assert abs(ta) < 1 << 287 and abs(tb) < 1 << 287
        a, b = ta >> K, tb >> K
        if a < 0:
            a, f0, g0 = -a, -f0, -g0
        if b < 0:
            b, f1, g1 = -b, -f1, -g1
        assert a < 1 << 254 and b < 1 << 254
        tu, tv = u * f0 + v * g0, u * f1 + v * g1
        tu = (tu + ((tu * minv) % (1 << K)) * m) >> K
        tv = (tv + ((tv * minv) % (1 << K)) * m) >> K
        assert -2 * m < tu < 3 * m and -2 * m < tv < 3 * m
        u, v = tu % m, tv % m
    return a, b, v


def _hard_inputs(m, rng, n_random):
    fib = [1, 2]
    while fib[-1] < m:
        fib.append(fib[-1] + fib[-2])
    ys = [1, 2, 3, m - 1, m - 2, (m - 1) // 2, (m + 1) // 2, (1 << 253) - 1, 1 << 253, (1 << 62) - 1, 1 << 62]
    ys += [f for f in fib[-10:] if f < m] + [1 << k for k in range(254)]
    ys += [rng.randrange(1, m) for _ in range(n_random)]
    ys += [rng.randrange(1, 1 << rng.randrange(1, 254)) for _ in range(n_random // 2)]
    return ys


@pytest.mark.parametrize("m", [bn.P, bn.R], ids=["p", "r"])
def test_binary_gcd_finishes_in_17_rounds(m):
    assert -(-(2 * m.bit_length() - 1) // K) == ROUNDS
    rng = random.Random(51)
    for y in _hard_inputs(m, rng, 600):
        a, b, v = _bgcd(y, m)
        assert (a, b) == (0, 1), y
        assert v == pow(y, -1, m), y
    # rounds after convergence leave the state unchanged
    a, b, v = _bgcd(12345, m, rounds=ROUNDS + 4)
    assert (a, b, v) == (0, 1, pow(12345, -1, m))


def _limbs(x):
    return [(x >> (32 * j)) & M32 for j in range(8)]


def _sliced_mont(a, b, p):
    inv = (-pow(p, -1, 1 << 32)) % (1 << 32)
    A, B, Pl = _limbs(a), _limbs(b), _limbs(p)
    t, c1, c2 = [0] * 8, [0] * 8, [0] * 8
    for i in range(8):
        lo = [0] * 8
        m = ((A[i] * B[0] + t[0] + c1[0] + c2[0]) & M32) * inv & M32
        for j in range(8):
            u = A[i] * B[j] + t[j] + c1[j]
            assert u < 1 << 64
            v = m * Pl[j] + (u & M32) + c2[j]
            assert v < 1 << 64
            c1[j], c2[j], lo[j] = u >> 32, v >> 32, v & M32
        assert lo[0] == 0
        t = lo[1:] + [0]
    s = [t[j] + c1[j] + c2[j] for j in range(8)]
    assert all(x >> 32 <= 2 for x in s)
    total = sum(x << (32 * j) for j, x in enumerate(s))
    assert total < 2 * p
    return total % p


@pytest.mark.parametrize("p", [bn.P, bn.R], ids=["p", "r"])
def test_sliced_product_bounds(p):
    rng = random.Random(52)
    rinv = pow(1 << 256, -1, p)
    edge = [0, 1, 2, p - 1, p - 2, (p - 1) // 2, M32, 1 << 253]
    pairs = [(x, y) for x in edge for y in edge] + [(rng.randrange(p), rng.randrange(p)) for _ in range(2000)]
    for x, y in pairs:
        assert _sliced_mont(x, y, p) == x * y * rinv % p


def test_carry_lookahead_identity():
    """Exhaustive over every (generate, propagate) pattern of eight limbs that never sets
    both bits of one limb: the lookahead equals the ripple."""
    for codes in itertools.product((0, 1, 2), repeat=8):  # 0 none, 1 generate, 2 propagate
        G = sum(1 << j for j, c in enumerate(codes) if c == 1)
        P = sum(1 << j for j, c in enumerate(codes) if c == 2)
        carry, ripple = 0, []
        for c in codes:
            ripple.append(carry)
            carry = 1 if c == 1 else (carry if c == 2 else 0)
        S = (G | P) + G
        assert [((S ^ P) >> j) & 1 for j in range(8)] == ripple
        assert (S >> 8) & 1 == carry


def test_sliced_point_formula_arrangements():
    """The XYZZ doubling and addition exactly as sliced.cuh arranges them (2X and 3X
    first, so that M = X 3X, 2S = 2X V and 3S = 3X V are products, X3 = M^2 - 2S and
    S - X3 = 3S - M^2; the addition's 2Q = 2U1 PP, X3 = (R^2 - PPP) - 2Q and
    Q - X3 = 3Q - (R^2 - PPP)) give the oracle's affine doubling and addition on random
    points in random XYZZ representations."""
    P = bn.P

    def dbl(X, Y, ZZ, ZZZ):
        U, X2 = 2 * Y % P, 2 * X % P
        X3x = (X2 + X) % P
        V, M = U * U % P, X * X3x % P
        W, MM, S2, S3 = U * V % P, M * M % P, X2 * V % P, X3x * V % P
        X3, SX = (MM - S2) % P, (S3 - MM) % P
        return X3, (M * SX - W * Y) % P, V * ZZ % P, W * ZZZ % P

    def add(p, q):
        X1, Y1, ZZ1, ZZZ1 = p
        X2, Y2, ZZ2, ZZZ2 = q
        U1, U2, S1, S2 = X1 * ZZ2 % P, X2 * ZZ1 % P, Y1 * ZZZ2 % P, Y2 * ZZZ1 % P
        Pd, R, U1x2 = (U2 - U1) % P, (S2 - S1) % P, 2 * U1 % P
        PP, RR, Z2, Z3 = Pd * Pd % P, R * R % P, ZZ1 * ZZ2 % P, ZZZ1 * ZZZ2 % P
        PPP, Q, ZZ3, Q2 = Pd * PP % P, U1 * PP % P, Z2 * PP % P, U1x2 * PP % P
        A, Q3 = (RR - PPP) % P, (Q + Q2) % P
        X3, QX = (A - Q2) % P, (Q3 - A) % P
        return X3, (R * QX - S1 * PPP) % P, ZZ3, Z3 * PPP % P

    def affine(pt):
        X, Y, ZZ, ZZZ = pt
        return X * pow(ZZ, -1, P) % P, Y * pow(ZZZ, -1, P) % P

    def xyzz(A, z):
        return A[0] * z * z % P, A[1] * z * z * z % P, z * z % P, z * z * z % P

    rng = random.Random(53)
    for _ in range(60):
        A = bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R))
        B = bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R))
        a, b = xyzz(A, rng.randrange(1, P)), xyzz(B, rng.randrange(1, P))
        assert affine(dbl(*a)) == bn.g1_add(A, A)
        assert affine(add(a, b)) == bn.g1_add(A, B)
