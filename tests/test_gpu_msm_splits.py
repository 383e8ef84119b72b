"""The endomorphism splits of the variable-base MSMs at their boundaries, on the GPU.

zkvc_msm_g1 splits every scalar as k = k1 + k2 lambda (mod r) with the GLV lattice
(phi(x, y) = (beta x, y) acts on G1 as lambda, a cube root of unity mod r), and
zkvc_msm_g2 splits it as k = k1 + k2 lambda2 with lambda2 = p mod r (psi, the twisted
Frobenius, acts on G2 as p).  Both splits run in the MSM's prep kernel, on every scalar.
Here the scalars are the values where a split can go wrong: 0, 1, r - 1, the
eigenvalues themselves and their neighbours, exact multiples m lambda2 and m lambda2 +- 1
(where the quotient estimate needs its correction), the rounding boundaries of the GLV
lattice (t r / b for the basis entries b), and powers of two around 2^127.  Each scalar
is checked alone (one point, the smallest window) and all together in one MSM over
distinct points, against the oracle's scalar multiplication and naive MSM.  Then the
scalars outside [0, r) that the prep kernels reduce mod r (up to 2^256 - 1), and the
degenerate MSMs: no points, zero scalars, a point and its negative, points at
infinity."""
import random

import pytest

from oracle import bn254 as bn
from tests import _util
from tests.test_glv_constants import _consts as _glv_consts

pytestmark = pytest.mark.gpu

R = bn.R


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _cube_roots_of_unity():
    """The two primitive cube roots of unity mod r, from the mathematics (r = 1 mod 3)."""
    out = set()
    for g in range(2, 50):
        w = pow(g, (R - 1) // 3, R)
        if w != 1:
            out.update({w, w * w % R})
        if len(out) == 2:
            return sorted(out)
    raise AssertionError("no cube root of unity found")


def _around(values, spread=(-1, 0, 1)):
    return [(v + d) % R for v in values for d in spread]


def _g1_edges():
    roots = _cube_roots_of_unity()
    ks = [0, 1, 2, R - 1, R - 2, R // 2, (R + 1) // 2]
    ks += _around(roots + [R - w for w in roots])
    ks += _around([1 << 126, 1 << 127, 1 << 128, 1 << 253])
    _, _, c = _glv_consts()
    for den in (c["GLV_B1"], c["GLV_B2"]):
        for t in (1, 2, 5):
            ks += _around([(t * R) // abs(den)])
    return sorted(set(ks))


def _g2_edges():
    lam2 = bn.P % R
    top = (R - 1) // lam2
    ks = [0, 1, 2, R - 1, R - 2, R // 2]
    ks += _around([lam2, R - lam2, lam2 * lam2 % R])
    ks += _around([m * lam2 for m in (2, 3, 1 << 64, top - 1, top)])
    ks += _around([1 << 126, 1 << 127, 1 << 128, 1 << 253])
    return sorted(set(k for k in ks if 0 <= k < R))


def _check(nv, group, ks, seed):
    rng = random.Random(seed)
    if group == 1:
        mul, msm, enc, rows, call = bn.g1_mul, bn.g1_msm, bn.g1_bytes, _util.g1_rows, nv.zkvc_msm_g1
        gen = bn.G1_GEN
    else:
        mul, msm, enc, rows, call = bn.g2_mul, bn.g2_msm, bn.g2_bytes, _util.g2_rows, nv.zkvc_msm_g2
        gen = bn.G2_GEN
    P = mul(gen, rng.randrange(1, R))
    Pd = _util.to_cuda(rows([P]))
    for k in ks:
        got = call(Pd, _util.to_cuda(_util.ints_to_u8([k])))
        assert got == enc(mul(P, k)), hex(k)
    pts = [mul(gen, rng.randrange(1, R)) for _ in ks]
    got = call(_util.to_cuda(rows(pts)), _util.to_cuda(_util.ints_to_u8(ks)))
    assert got == enc(msm(pts, ks))


def test_g1_glv_split_boundaries(nv):
    ks = _g1_edges()
    assert len(ks) > 40
    _check(nv, 1, ks, 11)


def test_g2_psi_split_boundaries(nv):
    ks = _g2_edges()
    assert len(ks) > 30
    _check(nv, 2, ks, 12)


@pytest.mark.parametrize("group", [1, 2])
def test_scalars_above_r_are_reduced(nv, group):
    rng = random.Random(13 + group)
    mul, enc, rows, call, gen = ((bn.g1_mul, bn.g1_bytes, _util.g1_rows, nv.zkvc_msm_g1, bn.G1_GEN) if group == 1
                                 else (bn.g2_mul, bn.g2_bytes, _util.g2_rows, nv.zkvc_msm_g2, bn.G2_GEN))
    P = mul(gen, rng.randrange(1, R))
    Pd = _util.to_cuda(rows([P]))
    top = (1 << 256) - 1
    for k in (R, R + 1, 2 * R - 1, 5 * R + 3, top - 1, top):
        assert k < 1 << 256
        assert call(Pd, _util.to_cuda(_util.ints_to_u8([k]))) == enc(mul(P, k % R)), hex(k)


@pytest.mark.parametrize("group", [1, 2])
def test_degenerate_msms(nv, group):
    import torch
    rng = random.Random(17 + group)
    if group == 1:
        mul, neg, msm, enc, rows, call, gen, width = (bn.g1_mul, bn.g1_neg, bn.g1_msm, bn.g1_bytes, _util.g1_rows,
                                                      nv.zkvc_msm_g1, bn.G1_GEN, 64)
    else:
        mul, neg, msm, enc, rows, call, gen, width = (bn.g2_mul, bn.g2_neg, bn.g2_msm, bn.g2_bytes, _util.g2_rows,
                                                      nv.zkvc_msm_g2, bn.G2_GEN, 128)
    empty = call(torch.empty((0, width), dtype=torch.uint8, device="cuda"),
                 torch.empty((0, 32), dtype=torch.uint8, device="cuda"))
    assert empty == enc(None) == bytes(width)
    P, Q = mul(gen, rng.randrange(1, R)), mul(gen, rng.randrange(1, R))
    cases = [
        ([P, Q], [0, 0]),                         # zero scalars
        ([P, neg(P)], [9, 9]),                    # cancellation
        ([P, Q], [5, R - 5]),                     # k P - k Q
        ([None, None], [3, 4]),                   # points at infinity only
        ([P] * 33, [R - 1] * 33),                 # one bucket, every term negative
    ]
    for pts, ks in cases:
        got = call(_util.to_cuda(rows(pts)), _util.to_cuda(_util.ints_to_u8(ks)))
        assert got == enc(msm(pts, ks)), (len(pts), ks[:2])
