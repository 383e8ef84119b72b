"""Tensor-core witness matmul Y = X W (int8 x int8 -> int32) against the exact integer
product: the oracle's matmul on small shapes, numpy's int64 matmul (the same definition,
a library routine) on the large ones.  Shapes cover a single element, ragged tails in all
three dimensions (tiles are 128 columns of Y by 64 rows, K in tiles of 64 and exactness
passes of 256), several passes, and the largest shape of the batched mix; the extreme
values (every product 2^14, all of one sign) check that the fp32 passes stay exact."""
import numpy as np
import pytest

from oracle import crpc
from paper_2504_12217_gb300 import inputs
from tests import _util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _gpu(nv, X, W):
    import torch
    return nv.zkvc_matmul_i8(torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()


SMALL = [(1, 1, 1), (4, 16, 8), (5, 17, 33), (2, 65, 3), (3, 300, 2), (64, 64, 128), (65, 1, 129)]


@pytest.mark.parametrize("shape", SMALL)
def test_matmul_small_against_oracle(nv, shape):
    a, n, b = shape
    X, W = inputs.matrices(4000 + a * 7 + n * 3 + b, a, n, b)
    got = _gpu(nv, X, W)
    want = crpc.matmul_int(X.astype(int).tolist(), W.astype(int).tolist())
    assert got.tolist() == want


LARGE = [(49, 320, 512), (130, 257, 129), (197, 768, 3072), (3, 1500, 7), (70, 1024, 200)]


@pytest.mark.parametrize("shape", LARGE)
def test_matmul_large_exact(nv, shape):
    a, n, b = shape
    X, W = inputs.matrices(5000 + a + n + b, a, n, b)
    got = _gpu(nv, X, W)
    want = X.astype(np.int64) @ W.astype(np.int64)
    assert got.dtype == np.int32 and np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("xv,wv", [(-128, -128), (-128, 127), (127, 127)])
def test_matmul_extremes(nv, xv, wv):
    a, n, b = 66, 1100, 130
    X = np.full((a, n), xv, dtype=np.int8)
    W = np.full((n, b), wv, dtype=np.int8)
    got = _gpu(nv, X, W)
    assert (got.astype(np.int64) == n * xv * wv).all()
    # an alternating pattern: partial sums cross zero inside each pass
    X2 = np.where((np.arange(n) % 2) == 0, -128, 127).astype(np.int8)[None, :].repeat(a, 0)
    got2 = _gpu(nv, X2, W)
    assert np.array_equal(got2.astype(np.int64), X2.astype(np.int64) @ W.astype(np.int64))


def test_matmul_rejects_bad_arguments(nv):
    import torch
    X = torch.zeros((2, 3), dtype=torch.int8, device="cuda")
    W = torch.zeros((4, 2), dtype=torch.int8, device="cuda")
    with pytest.raises(ValueError):
        nv.zkvc_matmul_i8(X, W)
    with pytest.raises(nv.ZkvcError):
        nv.check(nv.lib().zkvc_matmul_i8(None, None, None, 1, 1, 1, None))
