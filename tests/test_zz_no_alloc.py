"""The allocation-free G1 MSM entry point (for callers that cannot allocate device
memory) gives the same result as the workspace-based zkvc_msm_g1, call after call.

Collected last on purpose, so that a failure here leaves every other test already run."""
import random

import pytest

from oracle import bn254 as bn
from tests import _util

pytestmark = pytest.mark.gpu


def _points(rng, n):
    """n points with cheap oracle construction: an arithmetic progression b G + i d G."""
    P = bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R))
    D = bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R))
    pts = []
    for _ in range(n):
        pts.append(P)
        P = bn.g1_add(P, D)
    return pts


def test_noalloc_matches_workspace_msm_twice():
    import torch
    assert torch.cuda.is_available()
    nv = _util.native()
    rng = random.Random(2024)
    for n in (nv.ZKVC_MSM_NOALLOC_MAX_POINTS, 777):        # two calls in a row, different sizes
        pts = _points(rng, n)
        sc = [rng.randrange(bn.R) for _ in range(n)]
        sc[0] = 0
        P = _util.to_cuda(_util.g1_rows(pts))
        S = _util.to_cuda(_util.ints_to_u8(sc))
        got = nv.zkvc_msm_g1_noalloc(P, S)
        assert got == nv.zkvc_msm_g1(P, S)
        assert got != bytes(64)


def test_noalloc_matches_oracle_msm():
    """16 points: the allocation-free MSM equals the oracle's naive sum of scalar
    multiples (independent of the library's MSM code), twice in a row."""
    import torch
    assert torch.cuda.is_available()
    nv = _util.native()
    rng = random.Random(16)
    for _ in range(2):
        pts = [bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R)) for _ in range(16)]
        sc = [rng.randrange(bn.R) for _ in range(16)]
        sc[3] = bn.R - 1
        got = nv.zkvc_msm_g1_noalloc(_util.to_cuda(_util.g1_rows(pts)), _util.to_cuda(_util.ints_to_u8(sc)))
        assert got == bn.g1_bytes(bn.g1_msm(pts, sc))


def test_noalloc_rejects_oversize():
    import torch
    nv = _util.native()
    n = nv.ZKVC_MSM_NOALLOC_MAX_POINTS + 1
    P = torch.zeros((n, 64), dtype=torch.uint8, device="cuda")
    S = torch.zeros((n, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(nv.ZkvcError) as e:
        nv.zkvc_msm_g1_noalloc(P, S)
    assert e.value.code == nv.ZKVC_EINVAL
