"""The library's host-side GLV split (zkvc_glv_split, used by the chain-mode prover for s
and r) against the mathematics, without a GPU: k1 + k2 lambda = k (mod r) and
|k1|, |k2| < 2^127 for random scalars and the edge cases 0, 1, r - 1, lambda, r - lambda,
2^253 and values near the rounding boundaries of the lattice basis.  lambda is the cube
root of unity mod r that acts as phi(x, y) = (beta x, y) on G1 (checked against the
oracle's group law in test_glv_constants.py)."""
import random

from oracle import bn254 as bn
from tests import _util
from tests.test_glv_constants import _consts


def test_split_reproduces_k_with_short_halves():
    nv = _util.native()
    lam, _, c = _consts()
    rng = random.Random(41)
    ks = [0, 1, 2, 3, bn.R - 1, bn.R - 2, bn.R // 2, (bn.R + 1) // 2, 1 << 253, lam, bn.R - lam, (lam * 2) % bn.R]
    # near multiples of r / b: where the rounded coefficients change
    for den in (c["GLV_B1"], c["GLV_B2"]):
        for t in range(1, 6):
            base = (t * bn.R) // den
            ks += [max(0, min(bn.R - 1, base + d)) for d in (-1, 0, 1)]
    ks += [rng.randrange(bn.R) for _ in range(3000)]
    for k in ks:
        k1, k2 = nv.zkvc_glv_split(k)
        assert (k1 + k2 * lam - k) % bn.R == 0, k
        assert abs(k1) < 1 << 127 and abs(k2) < 1 << 127, k


def test_null_pointer_is_rejected():
    nv = _util.native()
    assert nv.lib().zkvc_glv_split(None, None) == nv.ZKVC_EINVAL
