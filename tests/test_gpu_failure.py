"""Failure paths on the GPU, made without faulting it.

* Bounded device waits: the tensor-core witness matmul's first mbarrier wait is told to
  give up at once (zkvc_set_device_wait_limit_ns(0)); the kernel must flag the timeout,
  wait for its own MMAs with the full limit, free its tensor memory and return, and the
  call must report ZKVC_ETIMEOUT; with the limit restored the same context computes the
  right product and the right proof.
* Unsatisfiable statements: zkvc_prove_claimed proves a claimed Y; the true X W gives the
  same proof as zkvc_prove, a Y off by one in a single entry is rejected with
  ZKVC_EUNSAT, by the PSQ check of the CRPC + PSQ circuit and by the quotient check
  (h_(N-1) != 0) of a circuit without prefix sums."""
import numpy as np
import pytest

from oracle import crpc, groth16 as og
from paper_2504_12217_gb300 import inputs
from tests import _util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def test_device_wait_timeout_reported_and_recovered(nv):
    import torch
    rng = np.random.default_rng(5)
    X = rng.integers(-128, 128, size=(70, 300), dtype=np.int8)
    W = rng.integers(-128, 128, size=(300, 200), dtype=np.int8)
    Xd, Wd = torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda()
    a, n, b = 5, 7, 3
    inst = inputs.instance(4242, (a, n, b))
    pk, _ = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    Xs, Ws = torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda()
    try:
        nv.zkvc_set_device_wait_limit_ns(0)
        for _ in range(2):
            with pytest.raises(nv.ZkvcError) as e:
                nv.zkvc_matmul_i8(Xd, Wd)
            assert e.value.code == nv.ZKVC_ETIMEOUT
        with pytest.raises(nv.ZkvcError) as e:
            nv.zkvc_prove(pk, Xs, Ws, inputs.to_bytes32(inst["rs"]))
        assert e.value.code == nv.ZKVC_ETIMEOUT
    finally:
        nv.zkvc_set_device_wait_limit_ns(200_000_000)
    torch.cuda.synchronize()
    Y = nv.zkvc_matmul_i8(Xd, Wd)
    assert np.array_equal(Y.cpu().numpy(), X.astype(np.int64) @ W.astype(np.int64))
    proof, _ = nv.zkvc_prove(pk, Xs, Ws, inputs.to_bytes32(inst["rs"]))
    X_, W_ = inst["X"].astype(int).tolist(), inst["W"].astype(int).tolist()
    cf, _ = og.closed_form_proof(crpc.Shape(a, n, b), inst["toxic"], X_, W_, *inst["rs"])
    assert proof == og.proof_bytes(cf)


@pytest.mark.parametrize("circuit", [None, "vanilla"])
def test_claimed_product(nv, circuit):
    import torch
    a, n, b = 4, 9, 6
    inst = inputs.instance(777, (a, n, b))
    toxic = inputs.to_bytes32(inst["toxic"])
    if circuit is None:
        pk, vk = nv.zkvc_setup(a, n, b, toxic)
    else:
        pk, vk = nv.zkvc_setup_circuit(a, n, b, circuit, "xy", toxic)
    Xd, Wd = torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda()
    rs = inputs.to_bytes32(inst["rs"])
    Ytrue = inst["X"].astype(np.int64) @ inst["W"].astype(np.int64)
    Yd = torch.from_numpy(Ytrue.astype(np.int32)).cuda()
    proof = nv.zkvc_prove_claimed(pk, Xd, Wd, Yd, rs)
    direct, _ = nv.zkvc_prove(pk, Xd, Wd, rs)
    assert proof == direct
    assert nv.zkvc_verify(vk, inst["X"], Ytrue.astype(np.int32), proof)
    assert np.array_equal(Yd.cpu().numpy(), Ytrue)        # the claimed Y is only read
    for (i, j) in [(0, 0), (a - 1, b - 1), (2, 3)]:
        bad = Ytrue.astype(np.int32).copy()
        bad[i, j] += 1
        with pytest.raises(nv.ZkvcError) as e:
            nv.zkvc_prove_claimed(pk, Xd, Wd, torch.from_numpy(bad).cuda(), rs)
        assert e.value.code == nv.ZKVC_EUNSAT
        assert ("PSQ" in str(e.value)) == (circuit is None)
        if circuit is not None:
            assert "quotient" in str(e.value)
