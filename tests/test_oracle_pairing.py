"""Pins of the oracle pairing: the Fp12 representation is a field containing Fp2, and
the pairing is bilinear, non-degenerate and lands in the order-r subgroup."""
import random

from oracle import bn254 as bn
from oracle import pairing as pr


def test_fp2_embeds_multiplicatively():
    rng = random.Random(1)
    for _ in range(5):
        a = (rng.randrange(bn.P), rng.randrange(bn.P))
        b = (rng.randrange(bn.P), rng.randrange(bn.P))
        assert pr.f12_mul(pr.fp2_to_f12(a), pr.fp2_to_f12(b)) == pr.fp2_to_f12(bn.f2_mul(a, b))
    # i^2 = -1 in the image
    i = pr.fp2_to_f12((0, 1))
    assert pr.f12_mul(i, i) == pr.f12([bn.P - 1])
    # w^6 = xi
    w = pr.f12([0, 1])
    assert pr.f12_pow(w, 6) == pr.fp2_to_f12(bn.XI)


def test_f12_inverse():
    rng = random.Random(2)
    for _ in range(3):
        a = pr.f12([rng.randrange(bn.P) for _ in range(12)])
        assert pr.f12_mul(a, pr.f12_inv(a)) == pr.F12_ONE


def test_untwist_lands_on_curve():
    Qx, Qy = pr.untwist(bn.G2_GEN)
    lhs = pr.f12_mul(Qy, Qy)
    rhs = pr.f12_add(pr.f12_mul(pr.f12_mul(Qx, Qx), Qx), pr.f12([3]))
    assert lhs == rhs


def test_bilinear_nondegenerate():
    rng = random.Random(3)
    a, b = rng.randrange(1, 1 << 64), rng.randrange(1, 1 << 64)
    e = pr.pairing(bn.G1_GEN, bn.G2_GEN)
    assert e != pr.F12_ONE
    assert pr.f12_pow(e, bn.R) == pr.F12_ONE
    eab = pr.pairing(bn.g1_mul(bn.G1_GEN, a), bn.g2_mul(bn.G2_GEN, b))
    assert eab == pr.f12_pow(e, a * b)
    # additivity in the first argument
    P1 = bn.g1_mul(bn.G1_GEN, 5)
    P2 = bn.g1_mul(bn.G1_GEN, 11)
    assert pr.f12_mul(pr.pairing(P1, bn.G2_GEN), pr.pairing(P2, bn.G2_GEN)) == \
        pr.pairing(bn.g1_add(P1, P2), bn.G2_GEN)


def test_product_check():
    P1 = bn.g1_mul(bn.G1_GEN, 7)
    Q1 = bn.g2_mul(bn.G2_GEN, 3)
    P2 = bn.g1_mul(bn.G1_GEN, 21)
    assert pr.pairing_product_is_one([(P1, Q1), (bn.g1_neg(P2), bn.G2_GEN)])
    assert not pr.pairing_product_is_one([(P1, Q1), (bn.g1_neg(P1), bn.G2_GEN)])
