"""GPU parity of the chain-mode prover and of the proof server: every proof equals the
oracle's (small shapes) and the one-proof fold prover's; a request's result is the same
alone and in a mix of concurrent requests of other shapes, under every policy (the merge
policy proves queued requests together as one batch); memory admission never lets the
requests in flight exceed the budget; a request that can never fit, a bad key index and
a bad (r, s) are reported per request, also inside a merged batch; waits are bounded."""
import threading

import numpy as np
import pytest

from oracle import bn254 as bn
from oracle import crpc, groth16 as og
from paper_2504_12217_gb300 import inputs
from tests import _util

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (3, 2, 2), (5, 7, 3), (2, 33, 40), (4, 16, 8), (6, 40, 3)]


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


@pytest.fixture(scope="module")
def keys(nv):
    out = []
    for shape in SHAPES:
        toxic = inputs.setup_values(7000 + shape[0] * 1000 + shape[1] * 10 + shape[2])
        pk, vk = nv.zkvc_setup(*shape, inputs.to_bytes32(toxic))
        out.append((pk, vk, toxic))
    return out


def _request(seed, shape):
    X, W = inputs.matrices(seed, *shape)
    return X, W, inputs.prover_values(seed)


def _oracle(shape, toxic, X, W, rs):
    proof, Y = og.closed_form_proof(crpc.Shape(*shape), toxic, X.astype(int).tolist(), W.astype(int).tolist(), *rs)
    return og.proof_bytes(proof), Y


def test_chain_mode_matches_oracle_and_fold(nv, keys):
    import torch
    for k, shape in enumerate(SHAPES):
        pk, _, toxic = keys[k]
        for seed in (11, 12):
            X, W, rs = _request(seed * 100 + k, shape)
            Xd, Wd = torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda()
            pc, Yc = nv.zkvc_prove_mode(pk, nv.ZKVC_PROVE_CHAIN, Xd, Wd, inputs.to_bytes32(rs))
            pf, _ = nv.zkvc_prove_mode(pk, nv.ZKVC_PROVE_FOLD, Xd, Wd, inputs.to_bytes32(rs))
            eproof, eY = _oracle(shape, toxic, X, W, rs)
            assert pc == eproof and pf == eproof, (shape, seed)
            assert Yc.cpu().numpy().tolist() == eY
        assert nv.zkvc_prove_workspace_bytes_mode(pk, nv.ZKVC_PROVE_CHAIN) > 0


def test_chain_mode_config2(nv):
    """[49,320] x [320,512]: the chain prover's proof equals the closed-form proof."""
    import torch
    a, n, b = inputs.SHAPE_CFG2
    inst = inputs.instance(inputs.SEED_CFG[2], (a, n, b))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    proof, Y = nv.zkvc_prove_mode(pk, nv.ZKVC_PROVE_CHAIN, torch.from_numpy(inst["X"]).cuda(),
                                  torch.from_numpy(inst["W"]).cuda(), inputs.to_bytes32(inst["rs"]))
    X, W = inst["X"].astype(int).tolist(), inst["W"].astype(int).tolist()
    cf, _ = og.closed_form_proof(crpc.Shape(a, n, b), inst["toxic"], X, W, *inst["rs"])
    assert proof == og.proof_bytes(cf)
    assert nv.zkvc_verify(vk, inst["X"], Y.cpu().numpy(), proof)


@pytest.mark.parametrize("policy", [0, 1, 2, 3])
def test_server_mix_equals_alone(nv, keys, policy):
    """Requests of all shapes submitted from two threads at once; each result equals the
    oracle's proof and Y for the same inputs.  Under the merge policy one worker takes the
    first request alone and the rest queue behind it, so most are proven in merged batches."""
    srv = nv.Server([k[0] for k in keys], slots=1 if policy == 3 else 4, mem_budget=256 << 20, policy=policy)
    reqs = [(i % len(SHAPES), _request(900 + 31 * i + policy, SHAPES[i % len(SHAPES)])) for i in range(24)]
    tickets = [None] * len(reqs)

    def submit(lo, hi):
        for i in range(lo, hi):
            k, (X, W, rs) = reqs[i]
            tickets[i] = srv.submit(k, X, W, inputs.to_bytes32(rs))

    th = [threading.Thread(target=submit, args=(0, 12)), threading.Thread(target=submit, args=(12, 24))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i, (k, (X, W, rs)) in enumerate(reqs):
        status, proof, Y, times = srv.wait(tickets[i], k)
        assert status == nv.ZKVC_OK
        eproof, eY = _oracle(SHAPES[k], keys[k][2], X, W, rs)
        assert proof == eproof, (i, SHAPES[k])
        assert Y.tolist() == eY
        assert times["total_ms"] >= times["prove_ms"] >= 0
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["in_flight"] == 0 and st["queued"] == 0
    assert st["bytes_in_use"] == 0 and 0 < st["peak_bytes"] <= 256 << 20
    if policy == nv.ZKVC_SERVER_FOLD:
        assert st["chain_mode"] == 0
    if policy == nv.ZKVC_SERVER_CHAIN:
        assert st["chain_mode"] == len(reqs)
    if policy == nv.ZKVC_SERVER_MERGE:
        assert st["merged_requests"] >= 2 and st["merged_batches"] >= 1
    else:
        assert st["merged_requests"] == 0
    srv.close()


def test_server_merge_status_and_admission(nv, keys):
    """Merge policy: a bad (r, s) inside a merged batch fails its own request only; with a
    budget that holds one request of the largest shape (as a one-request batch), batches
    shrink to what fits and everything completes within the budget."""
    srv = nv.Server([k[0] for k in keys], slots=1, mem_budget=256 << 20, policy=nv.ZKVC_SERVER_MERGE)
    reqs = [(i % len(SHAPES), _request(700 + i, SHAPES[i % len(SHAPES)])) for i in range(12)]
    tickets = []
    for i, (k, (X, W, rs)) in enumerate(reqs):
        tickets.append(srv.submit(k, X, W, inputs.to_bytes32([bn.R, 1] if i == 7 else rs)))
    for i, (t, (k, (X, W, rs))) in enumerate(zip(tickets, reqs)):
        status, proof, _, _ = srv.wait(t, k)
        if i == 7:
            assert status == nv.ZKVC_EINVAL and proof is None
        else:
            assert status == nv.ZKVC_OK and proof == _oracle(SHAPES[k], keys[k][2], X, W, rs)[0], i
    assert srv.stats()["merged_requests"] >= 2
    srv.close()
    big = max(range(len(SHAPES)), key=lambda k: nv.zkvc_server_request_bytes(keys[k][0], nv.ZKVC_PROVE_FOLD))
    budget = 3 * nv.zkvc_server_request_bytes(keys[big][0], nv.ZKVC_PROVE_FOLD) + (1 << 20)
    srv = nv.Server([k[0] for k in keys], slots=2, mem_budget=budget, policy=nv.ZKVC_SERVER_MERGE)
    reqs = [(big, _request(750 + i, SHAPES[big])) for i in range(10)]
    tickets = [srv.submit(k, X, W, inputs.to_bytes32(rs)) for k, (X, W, rs) in reqs]
    for t, (k, (X, W, rs)) in zip(tickets, reqs):
        status, proof, _, _ = srv.wait(t, k)
        assert status == nv.ZKVC_OK and proof == _oracle(SHAPES[k], keys[k][2], X, W, rs)[0]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["bytes_in_use"] == 0 and st["peak_bytes"] <= budget
    srv.close()


def test_server_memory_admission(nv, keys):
    """A budget that holds one request of the largest shape at a time: everything still
    completes, one by one, and the peak stays within the budget."""
    big = max(range(len(SHAPES)), key=lambda k: nv.zkvc_server_request_bytes(keys[k][0], nv.ZKVC_PROVE_FOLD))
    budget = nv.zkvc_server_request_bytes(keys[big][0], nv.ZKVC_PROVE_FOLD) + (1 << 20)
    budget = max(budget, 1 << 20)
    srv = nv.Server([k[0] for k in keys], slots=4, mem_budget=budget, policy=nv.ZKVC_SERVER_FOLD)
    reqs = [(big, _request(50 + i, SHAPES[big])) for i in range(6)]
    tickets = [srv.submit(k, X, W, inputs.to_bytes32(rs)) for k, (X, W, rs) in reqs]
    for t, (k, (X, W, rs)) in zip(tickets, reqs):
        status, proof, _, _ = srv.wait(t, k)
        assert status == nv.ZKVC_OK and proof == _oracle(SHAPES[k], keys[k][2], X, W, rs)[0]
    assert srv.stats()["peak_bytes"] <= budget
    srv.close()


def test_server_rejections_and_timeouts(nv, keys):
    srv = nv.Server([k[0] for k in keys], slots=2, mem_budget=1 << 20, policy=nv.ZKVC_SERVER_ADAPTIVE)
    big = max(range(len(SHAPES)), key=lambda k: nv.zkvc_server_request_bytes(keys[k][0], nv.ZKVC_PROVE_CHAIN))
    assert nv.zkvc_server_request_bytes(keys[big][0], nv.ZKVC_PROVE_CHAIN) > 1 << 20
    X, W, rs = _request(3, SHAPES[big])
    t = srv.submit(big, X, W, inputs.to_bytes32(rs))
    status, proof, _, _ = srv.wait(t, big)
    assert status == nv.ZKVC_ENOMEM and proof is None
    with pytest.raises(nv.ZkvcError) as e:
        srv.submit(len(SHAPES), X, W, inputs.to_bytes32(rs))
    assert e.value.code == nv.ZKVC_EINVAL
    with pytest.raises(nv.ZkvcError) as e:
        srv.wait(123456, 0)
    assert e.value.code == nv.ZKVC_EINVAL
    srv.close()
    # a bad (r, s) fails its own request only; a zero-millisecond wait on a busy server
    # times out and the ticket stays valid
    srv = nv.Server([k[0] for k in keys], slots=2, mem_budget=256 << 20)
    k0 = 0
    Xa, Wa, rsa = _request(4, SHAPES[k0])
    bad = srv.submit(k0, Xa, Wa, inputs.to_bytes32([bn.R + 1, 2]))
    many = [srv.submit(3, *_request(60 + i, SHAPES[3])[:2], inputs.to_bytes32(rsa)) for i in range(8)]
    with pytest.raises(nv.ZkvcError) as e:
        srv.wait(many[-1], 3, timeout_ms=0)
    assert e.value.code == nv.ZKVC_ETIMEOUT
    status, _, _, _ = srv.wait(bad, k0)
    assert status == nv.ZKVC_EINVAL
    for t in many:
        assert srv.wait(t, 3)[0] == nv.ZKVC_OK
    srv.close()


@pytest.mark.parametrize("policy", [0, 3])
def test_server_config4_shapes(nv, policy):
    """Three [tokens, dim] x [dim, *] shapes of the served workload at full size, 12
    requests in flight together (merge policy: in merged batches of mixed shapes): each
    proof equals the one-proof prover's on its own."""
    import torch
    shapes = [(49, 192, 192), (64, 192, 768), (49, 320, 320)]
    pks = [nv.zkvc_setup(*s, inputs.to_bytes32(inputs.setup_values(8000 + i)))[0] for i, s in enumerate(shapes)]
    srv = nv.Server(pks, slots=1 if policy == 3 else 4, mem_budget=8 << 30, policy=policy)
    reqs = []
    for i in range(12):
        k = i % 3
        X, W = inputs.matrices(8100 + i, *shapes[k])
        reqs.append((k, X, W, inputs.to_bytes32(inputs.prover_values(8100 + i))))
    tickets = [srv.submit(k, X, W, rs) for k, X, W, rs in reqs]
    for t, (k, X, W, rs) in zip(tickets, reqs):
        status, proof, Y, _ = srv.wait(t, k)
        assert status == nv.ZKVC_OK
        alone, Ya = nv.zkvc_prove(pks[k], torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(), rs)
        assert proof == alone
        assert np.array_equal(Y, Ya.cpu().numpy())
    if policy == 3:
        assert srv.stats()["merged_requests"] >= 2
    srv.close()
