"""Pins of the oracle's BN254 parameters, fields and groups against facts fixed by the
mathematics of the curve (not by re-running the oracle's own formulas)."""
import random

from oracle import bn254 as bn


def test_moduli_prime_and_related():
    assert bn.is_probable_prime(bn.P)
    assert bn.is_probable_prime(bn.R)
    assert bn.P % 4 == 3
    # Hasse: #E(Fp) = p + 1 - t with the BN trace t = 6u^2 + 1, and it is the prime r
    assert bn.R == bn.P + 1 - (6 * bn.U**2 + 1)
    assert bn.P.bit_length() == 254 and bn.R.bit_length() == 254
    assert bn.R > 1 << 253


def test_known_decimal_moduli():
    # the decimal values printed with EIP-196/197 for alt_bn128
    assert bn.P == 21888242871839275222246405745257275088696311157297823662689037894645226208583
    assert bn.R == 21888242871839275222246405745257275088548364400416034343698204186575808495617


def test_g1_generator_order():
    assert bn.g1_on_curve(bn.G1_GEN)
    assert bn.g1_mul_noshortcut(bn.G1_GEN, bn.R) is None
    assert bn.g1_mul_noshortcut(bn.G1_GEN, bn.R - 1) == bn.g1_neg(bn.G1_GEN)


def test_g2_generator_order():
    assert bn.g2_on_curve(bn.G2_GEN)
    assert bn.g2_mul_noshortcut(bn.G2_GEN, bn.R) is None
    assert bn.g2_mul_noshortcut(bn.G2_GEN, bn.R + 1) == bn.G2_GEN


def test_tower_non_residue():
    # Fp6 = Fp2[v]/(v^3 - xi) and Fp12 = Fp6[w]/(w^2 - v) need xi to be neither a square
    # nor a cube in Fp2.
    q = bn.P * bn.P - 1
    assert bn.f2_pow(bn.XI, q // 2) != bn.F2_ONE
    assert bn.f2_pow(bn.XI, q // 3) != bn.F2_ONE
    # b' = 3/xi really is the twist coefficient: b' xi = 3
    assert bn.f2_mul(bn.B2, bn.XI) == (3, 0)


def test_fr_two_adicity_and_roots():
    assert (bn.R - 1) % (1 << 28) == 0 and ((bn.R - 1) >> 28) % 2 == 1
    # 5 is a quadratic non-residue, so 5^((r-1)/2^28) has order exactly 2^28
    assert pow(bn.FR_GEN, (bn.R - 1) // 2, bn.R) == bn.R - 1
    for logn in (1, 2, 7, 16, 20, 24, 28):
        n = 1 << logn
        w = bn.fr_root_of_unity(n)
        assert pow(w, n, bn.R) == 1
        assert pow(w, n // 2, bn.R) == bn.R - 1
    # the coset shift is outside every power-of-two subgroup: g^N != 1
    assert pow(bn.FR_GEN, 1 << 28, bn.R) != 1


def test_fr_from_int_negatives():
    assert bn.fr_from_int(-1) == bn.R - 1
    assert bn.fr_from_int(-128) == bn.R - 128
    assert bn.fr_from_int(127) == 127


def _affine_mul(Pt, k, add):
    acc = None
    for bit in bin(k)[2:]:
        acc = add(acc, acc)
        if bit == "1":
            acc = add(acc, Pt)
    return acc


def test_g1_mul_brute_force_small():
    acc = None
    for k in range(0, 40):
        assert bn.g1_mul(bn.G1_GEN, k) == acc
        acc = bn.g1_add(acc, bn.G1_GEN)


def test_g1_mul_against_affine_ladder():
    rng = random.Random(7)
    Q = bn.g1_mul(bn.G1_GEN, 123456789)
    for _ in range(5):
        k = rng.randrange(1, bn.R)
        ref = _affine_mul(Q, k, bn.g1_add)
        assert bn.g1_mul(Q, k) == ref
    # the -[r-k]P shortcut agrees with the plain ladder
    k = bn.R - 12345
    assert bn.g1_mul(Q, k) == _affine_mul(Q, k, bn.g1_add)


def test_g2_mul_brute_force_and_ladder():
    acc = None
    for k in range(0, 12):
        assert bn.g2_mul(bn.G2_GEN, k) == acc
        acc = bn.g2_add(acc, bn.G2_GEN)
    rng = random.Random(8)
    for _ in range(2):
        k = rng.randrange(1, bn.R)
        assert bn.g2_mul(bn.G2_GEN, k) == _affine_mul(bn.G2_GEN, k, bn.g2_add)


def test_msm_brute_force_and_linearity():
    rng = random.Random(9)
    pts = [bn.g1_mul(bn.G1_GEN, rng.randrange(1, 1000)) for _ in range(6)]
    sc = [rng.randrange(0, 9) for _ in range(6)]
    brute = None
    for Pt, s in zip(pts, sc):
        for _ in range(s):
            brute = bn.g1_add(brute, Pt)
    assert bn.g1_msm(pts, sc) == brute
    s1 = [rng.randrange(bn.R) for _ in range(6)]
    s2 = [rng.randrange(bn.R) for _ in range(6)]
    both = [(x + y) % bn.R for x, y in zip(s1, s2)]
    assert bn.g1_msm(pts, both) == bn.g1_add(bn.g1_msm(pts, s1), bn.g1_msm(pts, s2))
    # negative (int8-style) scalars map through r - |v|
    neg = [bn.fr_from_int(-v) for v in sc]
    assert bn.g1_msm(pts, neg) == bn.g1_neg(brute)


def test_g2_msm_brute_force():
    rng = random.Random(10)
    pts = [bn.g2_mul(bn.G2_GEN, rng.randrange(1, 1000)) for _ in range(3)]
    sc = [3, 0, 5]
    brute = None
    for Pt, s in zip(pts, sc):
        for _ in range(s):
            brute = bn.g2_add(brute, Pt)
    assert bn.g2_msm(pts, sc) == brute


def test_serialisation_round_trip():
    Pt = bn.g1_mul(bn.G1_GEN, 99)
    Q = bn.g2_mul(bn.G2_GEN, 99)
    assert bn.g1_from_bytes(bn.g1_bytes(Pt)) == Pt
    assert bn.g2_from_bytes(bn.g2_bytes(Q)) == Q
    assert bn.g1_bytes(None) == bytes(64) and bn.g2_bytes(None) == bytes(128)
    assert bn.g1_bytes(bn.G1_GEN)[:32] == (1).to_bytes(32, "little")
