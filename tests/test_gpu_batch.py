"""GPU parity of the batched prover: every proof of a batch equals, byte for byte, the
oracle's proof of the same (pk, X, W, r, s) and the one-proof GPU prover's, whether the
batch runs eagerly, as a captured-and-replayed CUDA graph, or after autotuning; a second
call with new inputs through the same graph gives the new proofs; a bad instance is
reported per instance without disturbing the others.  The full-size case proves the
seeded 64-instance mix of [tokens, dim] x [dim, dim or 4 dim] shapes."""
import os

import numpy as np
import pytest

from oracle import bn254 as bn
from oracle import crpc, groth16 as og
from paper_2504_12217_gb300 import inputs
from tests import _util

pytestmark = pytest.mark.gpu

SMALL = [(1, 1, 1), (2, 1, 3), (3, 2, 2), (5, 7, 3), (2, 33, 40), (4, 16, 8), (3, 2, 2), (6, 40, 3)]


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _shape_seed(base, shape):
    a, n, b = shape
    return base ^ (a << 40) ^ (n << 20) ^ b


@pytest.fixture(scope="module")
def small_keys(nv):
    """GPU keys and toxic waste of the distinct small shapes (the two (3, 2, 2) instances
    share one key)."""
    keys = {}
    for shape in dict.fromkeys(SMALL):
        toxic = inputs.setup_values(_shape_seed(5000, shape))
        pk, vk = nv.zkvc_setup(*shape, inputs.to_bytes32(toxic))
        keys[shape] = (pk, vk, toxic)
    return keys


def _instances(seed0, shapes):
    out = []
    for i, shape in enumerate(shapes):
        seed = seed0 + 17 * i
        X, W = inputs.matrices(seed, *shape)
        out.append((X, W, inputs.prover_values(seed)))
    return out


def _cuda(arrs):
    import torch
    return [torch.from_numpy(a).cuda() for a in arrs]


def _oracle_proofs(small_keys, shapes, insts):
    """The oracle's proofs (closed form from the toxic waste, equal to its prove)."""
    res = []
    for shape, (X, W, rs) in zip(shapes, insts):
        toxic = small_keys[shape][2]
        proof, Y = og.closed_form_proof(crpc.Shape(*shape), toxic, X.astype(int).tolist(), W.astype(int).tolist(), *rs)
        res.append((og.proof_bytes(proof), Y))
    return res


@pytest.mark.parametrize("flags", [0, 2, 1])  # graph, eager, autotuned graph
def test_batch_small_shapes(nv, small_keys, flags):
    pks = [small_keys[s][0] for s in SMALL]
    batch = nv.Batch(pks, flags=flags)
    for call, seed0 in enumerate((100, 900)):
        insts = _instances(seed0 + flags, SMALL)
        Xs = _cuda([x for x, _, _ in insts])
        Ws = _cuda([w for _, w, _ in insts])
        rs = [inputs.to_bytes32(r) for _, _, r in insts]
        proofs, Ys = batch.prove(Xs, Ws, rs)
        expect = _oracle_proofs(small_keys, SMALL, insts)
        for i, ((eproof, eY), proof, Y) in enumerate(zip(expect, proofs, Ys)):
            assert Y.cpu().numpy().tolist() == eY, (call, i)
            assert proof == eproof, (call, i, SMALL[i])
        # the one-proof GPU prover agrees on the same inputs
        p0, _ = nv.zkvc_prove(pks[4], Xs[4], Ws[4], rs[4])
        assert p0 == proofs[4]
    if flags == 1:
        t = batch.get_tuning()
        assert t["main_chunk"] in (8, 16, 32, 64, 128, 256) and t["ntt_log_elems_per_block"] in (9, 10, 11)
    info = batch.info()
    assert info["count"] == len(SMALL) and info["device_bytes"] > 0
    assert (info["graph_launches"] > 0) == (flags != 2)


def test_batch_set_tuning_and_one_shot(nv, small_keys):
    pks = [small_keys[s][0] for s in SMALL]
    insts = _instances(333, SMALL)
    Xs = _cuda([x for x, _, _ in insts])
    Ws = _cuda([w for _, w, _ in insts])
    rs = [inputs.to_bytes32(r) for _, _, r in insts]
    expect = [p for p, _ in _oracle_proofs(small_keys, SMALL, insts)]
    batch = nv.Batch(pks)
    for tuning in ([64, 64, 8, 256, 32, 64, 11], [8, 256, 64, 64, 8, 128, 9]):
        batch.set_tuning(tuning)
        assert list(batch.get_tuning().values()) == tuning
        proofs, _ = batch.prove(Xs, Ws, rs)
        assert proofs == expect
    with pytest.raises(nv.ZkvcError):
        batch.set_tuning([4, 128, 16, 128, 8, 128, 10])  # chunk below the sized minimum
    proofs, _ = nv.zkvc_prove_batch(pks, Xs, Ws, rs)
    assert proofs == expect


def test_batch_bad_instance_is_isolated(nv, small_keys):
    pks = [small_keys[s][0] for s in SMALL]
    insts = _instances(444, SMALL)
    Xs = _cuda([x for x, _, _ in insts])
    Ws = _cuda([w for _, w, _ in insts])
    rs = [inputs.to_bytes32(r) for _, _, r in insts]
    rs[2] = inputs.to_bytes32([bn.R, 5])  # r = the group order: not canonical
    batch = nv.Batch(pks)
    with pytest.raises(nv.ZkvcError) as e:
        batch.prove(Xs, Ws, rs)
    assert e.value.code == nv.ZKVC_EINVAL
    proofs, _, status = batch.prove(Xs, Ws, rs, with_status=True)
    assert status[2] == nv.ZKVC_EINVAL and all(s == nv.ZKVC_OK for i, s in enumerate(status) if i != 2)
    expect = _oracle_proofs(small_keys, SMALL, insts)
    for i in range(len(SMALL)):
        if i != 2:
            assert proofs[i] == expect[i][0], i


def test_batch_rejects_bad_arguments(nv, small_keys):
    with pytest.raises(nv.ZkvcError):
        nv.Batch([])
    pk = small_keys[SMALL[0]][0]
    with pytest.raises(nv.ZkvcError):
        nv.Batch([pk], flags=8)


def _golden_batch64():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "closed_form_batch64.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        i, a, n, b, proof = line.split()
        out[int(i)] = ((int(a), int(n), int(b)), bytes.fromhex(proof))
    return out


def test_batch_config4_full(nv):
    """The seeded 64-instance mix at full size, through the autotuned captured graph:
    every proof equals the oracle's closed-form proof of its instance (tests/golden,
    written by tests/golden/make_closed_form.py from oracle/ alone), the graph replay
    reproduces them, every proof's Y equals X W, and the one-proof prover agrees."""
    import torch
    shapes = inputs.batch_shapes()
    gold = _golden_batch64()
    assert [gold[i][0] for i in range(len(shapes))] == shapes
    keys = {}
    for shape in dict.fromkeys(shapes):
        toxic = inputs.setup_values(_shape_seed(inputs.SEED_CFG[4], shape))
        keys[shape] = (nv.zkvc_setup(*shape, inputs.to_bytes32(toxic))[0], toxic)
    insts = [inputs.instance(inputs.SEED_CFG[4] + 1000 + i, s) for i, s in enumerate(shapes)]
    Xs = [torch.from_numpy(t["X"]).cuda() for t in insts]
    Ws = [torch.from_numpy(t["W"]).cuda() for t in insts]
    rs = [inputs.to_bytes32(t["rs"]) for t in insts]
    batch = nv.Batch([keys[s][0] for s in shapes], flags=nv.ZKVC_BATCH_AUTOTUNE)
    proofs, Ys = batch.prove(Xs, Ws, rs)
    for i in range(len(shapes)):
        assert proofs[i] == gold[i][1], (i, shapes[i])
    proofs2, _ = batch.prove(Xs, Ws, rs)  # graph replay
    assert proofs2 == proofs
    for i, s in enumerate(shapes):
        Yi = Ys[i].cpu().numpy()
        assert np.array_equal(Yi, insts[i]["X"].astype(np.int64) @ insts[i]["W"].astype(np.int64)), i
        p1, _ = nv.zkvc_prove(keys[s][0], Xs[i], Ws[i], rs[i])
        assert p1 == proofs[i], (i, s)
