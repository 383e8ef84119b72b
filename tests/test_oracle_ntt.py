"""Pins of the oracle NTT: the O(N^2) definition, the round trip, direct evaluation on
the coset, and the convolution theorem against schoolbook polynomial products."""
import random

from oracle import bn254 as bn
from oracle import ntt as nt

R = bn.R


def _rand(n, seed):
    rng = random.Random(seed)
    return [rng.randrange(R) for _ in range(n)]


def test_ntt_matches_dft():
    for logn in range(0, 9):
        n = 1 << logn
        a = _rand(n, logn)
        assert nt.ntt(a) == nt.dft(a, bn.fr_root_of_unity(n))


def test_round_trip():
    for logn in (1, 4, 10):
        a = _rand(1 << logn, 100 + logn)
        assert nt.intt(nt.ntt(a)) == a
        assert nt.coset_intt(nt.coset_ntt(a)) == a


def test_coset_is_evaluation_at_shifted_points():
    n = 16
    a = _rand(n, 5)
    w = bn.fr_root_of_unity(n)
    ev = nt.coset_ntt(a)
    for k in range(n):
        x = bn.FR_GEN * pow(w, k, R) % R
        assert ev[k] == nt.poly_eval(a, x)


def test_convolution_theorem():
    n = 32
    a = _rand(n // 2, 6) + [0] * (n // 2)
    b = _rand(n // 2, 7) + [0] * (n // 2)
    prod = nt.intt([x * y % R for x, y in zip(nt.ntt(a), nt.ntt(b))])
    ref = nt.poly_mul_schoolbook(a[: n // 2], b[: n // 2]) + [0]
    assert prod == ref


def test_special_inputs():
    n = 8
    assert nt.ntt([1] + [0] * (n - 1)) == [1] * n          # delta -> constant
    assert nt.ntt([1] * n) == [n] + [0] * (n - 1)          # constant -> delta
    assert nt.ntt([0] * n) == [0] * n
