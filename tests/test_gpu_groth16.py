"""GPU parity of Groth16 setup and prove for the CRPC + PSQ circuit against the oracle.

Keys and proofs are compared byte for byte (field and group results are exact).  Small
shapes compare every key entry and the naive oracle proof; the full [49,320]x[320,512]
workload compares the proof with the oracle's closed-form proof (computed from the toxic
waste in the exponent) and sampled key entries, each computed one by one."""
import random

import numpy as np
import pytest

from oracle import bn254 as bn
from oracle import crpc, groth16 as og
from paper_2504_12217_gb300 import inputs
from tests import _util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _mats(X, W):
    return X.astype(int).tolist(), W.astype(int).tolist()


def _gpu_prove(nv, pk, X, W, rs):
    import torch
    proof, Y = nv.zkvc_prove(pk, torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(), rs)
    return proof, Y.cpu().numpy()


def _check_keys(nv, pk, vk, opk, ovk, sh):
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_A, 0, len(opk.A)) == b"".join(bn.g1_bytes(p) for p in opk.A)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_B1, 0, len(opk.B1)) == b"".join(bn.g1_bytes(p) for p in opk.B1)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_B2, 0, len(opk.B2)) == b"".join(bn.g2_bytes(p) for p in opk.B2)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_L, 0, len(opk.L)) == b"".join(bn.g1_bytes(p) for p in opk.L)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_H, 0, len(opk.H)) == b"".join(bn.g1_bytes(p) for p in opk.H)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_ALPHA1, 0, 1) == bn.g1_bytes(opk.alpha1)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_BETA1, 0, 1) == bn.g1_bytes(opk.beta1)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_BETA2, 0, 1) == bn.g2_bytes(opk.beta2)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_DELTA1, 0, 1) == bn.g1_bytes(opk.delta1)
    assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_DELTA2, 0, 1) == bn.g2_bytes(opk.delta2)
    assert nv.zkvc_vk_export(vk, nv.ZKVC_VK_IC, 0, len(ovk.IC)) == b"".join(bn.g1_bytes(p) for p in ovk.IC)
    assert nv.zkvc_vk_export(vk, nv.ZKVC_VK_GAMMA2, 0, 1) == bn.g2_bytes(ovk.gamma2)
    assert nv.zkvc_vk_export(vk, nv.ZKVC_VK_ALPHA1, 0, 1) == bn.g1_bytes(ovk.alpha1)
    assert nv.zkvc_vk_export(vk, nv.ZKVC_VK_BETA2, 0, 1) == bn.g2_bytes(ovk.beta2)
    assert nv.zkvc_vk_export(vk, nv.ZKVC_VK_DELTA2, 0, 1) == bn.g2_bytes(ovk.delta2)


def test_config1_keys_and_proof(nv):
    """[4,16] x [16,8]: every key entry and the proof equal the oracle's."""
    seed = inputs.SEED_CFG[1]
    a, n, b = inputs.SHAPE_CFG1
    inst = inputs.instance(seed, (a, n, b))
    toxic, rs = inst["toxic"], inst["rs"]
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(toxic))
    sh = crpc.Shape(a, n, b)
    assert pk.log_domain == 7
    opk, ovk = og.setup(sh, toxic)
    _check_keys(nv, pk, vk, opk, ovk, sh)
    proof, Y = _gpu_prove(nv, pk, inst["X"], inst["W"], inputs.to_bytes32(rs))
    assert np.array_equal(Y, inst["X"].astype(np.int64) @ inst["W"].astype(np.int64))
    X, W = _mats(inst["X"], inst["W"])
    oproof, _, _ = og.prove(opk, X, W, *rs)
    assert proof == og.proof_bytes(oproof)
    assert og.verify(ovk, X, Y.tolist(), og.proof_from_bytes(proof))


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 3), (1, 5, 1), (3, 2, 2), (5, 7, 3), (2, 33, 40)])
def test_small_shapes_keys_and_proof(nv, shape):
    a, n, b = shape
    seed = 1000 + a * 100 + n * 10 + b
    inst = inputs.instance(seed, shape)
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    opk, ovk = og.setup(crpc.Shape(a, n, b), inst["toxic"])
    _check_keys(nv, pk, vk, opk, ovk, crpc.Shape(a, n, b))
    X, W = _mats(inst["X"], inst["W"])
    for rs in (inst["rs"], [0, 0], [bn.R - 1, 1]):
        proof, Y = _gpu_prove(nv, pk, inst["X"], inst["W"], inputs.to_bytes32(rs))
        oproof, oY, _ = og.prove(opk, X, W, *rs)
        assert Y.tolist() == oY
        assert proof == og.proof_bytes(oproof), rs


def test_extreme_matrices(nv):
    """All -128 entries give the largest |y| (n 2^14) and one bucket per MSM."""
    a, n, b = 3, 40, 5
    inst = inputs.instance(77, (a, n, b))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    sh = crpc.Shape(a, n, b)
    for fill in (-128, 127, 0):
        X = np.full((a, n), fill, dtype=np.int8)
        W = np.full((n, b), fill, dtype=np.int8)
        proof, Y = _gpu_prove(nv, pk, X, W, inputs.to_bytes32(inst["rs"]))
        cf, _ = og.closed_form_proof(sh, inst["toxic"], X.astype(int).tolist(), W.astype(int).tolist(), *inst["rs"])
        assert proof == og.proof_bytes(cf), fill


def test_config2_full_size(nv):
    """[49,320] x [320,512] (N = 2^16): proof equals the closed-form proof; key entries
    sampled across every query equal [scalar]G computed one by one."""
    a, n, b = inputs.SHAPE_CFG2
    inst = inputs.instance(inputs.SEED_CFG[2], (a, n, b))
    toxic, rs = inst["toxic"], inst["rs"]
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(toxic))
    assert pk.log_domain == 16
    proof, Y = _gpu_prove(nv, pk, inst["X"], inst["W"], inputs.to_bytes32(rs))
    assert np.array_equal(Y, inst["X"].astype(np.int64) @ inst["W"].astype(np.int64))
    sh = crpc.Shape(a, n, b)
    X, W = _mats(inst["X"], inst["W"])
    cf, _ = og.closed_form_proof(sh, toxic, X, W, *rs)
    assert proof == og.proof_bytes(cf)
    rng = random.Random(2)
    sizes = {"A": sh.n_public + 1, "B": n * b, "L": n * b + n - 1, "H": sh.domain - 1, "IC": sh.n_public + 1}
    qids = {"A": nv.ZKVC_Q_A, "B": nv.ZKVC_Q_B1, "L": nv.ZKVC_Q_L, "H": nv.ZKVC_Q_H}
    for q, size in sizes.items():
        idx = sorted(set([0, size - 1] + [rng.randrange(size) for _ in range(6)]))
        scal = og.pk_entry_scalars(sh, toxic, q, idx)
        for i, s in zip(idx, scal):
            if q == "IC":
                got = nv.zkvc_vk_export(vk, nv.ZKVC_VK_IC, i, 1)
            else:
                got = nv.zkvc_pk_export(pk, qids[q], i, 1)
            assert got == bn.g1_bytes(bn.g1_mul(bn.G1_GEN, s)), (q, i)
            if q == "B":
                assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_B2, i, 1) == bn.g2_bytes(bn.g2_mul(bn.G2_GEN, s))


def test_rejected_inputs(nv):
    a, n, b = 2, 3, 2
    inst = inputs.instance(5, (a, n, b))
    good = list(inst["toxic"])
    for bad in ([bn.R] + good[1:], good[:1] + [0] + good[2:], good[:5] + [1], good[:5] + [0]):
        with pytest.raises(nv.ZkvcError) as e:
            nv.zkvc_setup(a, n, b, inputs.to_bytes32(bad))
        assert e.value.code == nv.ZKVC_EINVAL
    with pytest.raises(nv.ZkvcError):
        nv.zkvc_setup(0, 3, 2, inputs.to_bytes32(good))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(good))
    with pytest.raises(nv.ZkvcError) as e:
        _gpu_prove(nv, pk, inst["X"], inst["W"], inputs.to_bytes32([bn.R, 1]))
    assert e.value.code == nv.ZKVC_EINVAL


def test_pk_save_load_and_verify(nv, tmp_path):
    """A reloaded proving key proves the same bytes; the library verifier accepts GPU
    proofs and rejects a tampered statement; corrupt key files are refused."""
    a, n, b = 3, 9, 6
    inst = inputs.instance(4242, (a, n, b))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    rs = inputs.to_bytes32(inst["rs"])
    proof, Y = _gpu_prove(nv, pk, inst["X"], inst["W"], rs)
    assert nv.zkvc_verify(vk, inst["X"], Y, proof)
    Yt = Y.copy()
    Yt[0, 0] ^= 1
    assert not nv.zkvc_verify(vk, inst["X"], Yt, proof)
    path = tmp_path / "k.pk"
    nv.zkvc_pk_save(pk, str(path))
    pk2 = nv.zkvc_pk_load(str(path))
    assert pk2.shape == pk.shape
    proof2, _ = _gpu_prove(nv, pk2, inst["X"], inst["W"], rs)
    assert proof2 == proof
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 1
    bad = tmp_path / "bad.pk"
    bad.write_bytes(bytes(raw))
    with pytest.raises(nv.ZkvcError) as e:
        nv.zkvc_pk_load(str(bad))
    assert e.value.code == nv.ZKVC_EIO


def test_verifier_accepts_config2_gpu_proof(nv):
    a, n, b = inputs.SHAPE_CFG2
    inst = inputs.instance(inputs.SEED_CFG[2], (a, n, b))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    proof, Y = _gpu_prove(nv, pk, inst["X"], inst["W"], inputs.to_bytes32(inst["rs"]))
    assert nv.zkvc_verify(vk, inst["X"], Y, proof)
    bad = proof[:192] + bn.g1_bytes(bn.g1_add(bn.g1_from_bytes(proof[192:]), bn.G1_GEN))
    assert not nv.zkvc_verify(vk, inst["X"], Y, bad)


def test_autotuned_and_imposed_tuning_prove_same_bytes(nv):
    """Chunk sizes and NTT blocks change only the launch shape: autotuned, imposed and
    default settings give the same proof, in both prover modes."""
    import torch
    a, n, b = 5, 40, 33
    inst = inputs.instance(555, (a, n, b))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    Xd, Wd = torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda()
    rs = inputs.to_bytes32(inst["rs"])
    p0, _ = nv.zkvc_prove(pk, Xd, Wd, rs)
    chosen = nv.zkvc_pk_autotune(pk, Xd, Wd, rs, mode=nv.ZKVC_PROVE_AUTO)
    assert all(c in (0, 2, 4, 8, 16, 32, 64) for c in chosen[:4]) and chosen[4] in (0, 8, 9, 11)
    assert chosen[5] in (0, 1, 2) and all(c in (0, 1) for c in chosen[6:])
    assert nv.zkvc_pk_get_tuning(pk) == chosen
    assert nv.zkvc_prove(pk, Xd, Wd, rs)[0] == p0
    for tuning in ([2, 2, 2, 2, 8, 1, 0, 1, 1, 0], [64, 1, 3, 7, 11, 2, 1, 0, 0, 1], [0, 0, 0, 0, 9, 1, 1, 1, 1, 1]):
        nv.zkvc_pk_set_tuning(pk, tuning)
        assert nv.zkvc_pk_get_tuning(pk) == tuning
        assert nv.zkvc_prove(pk, Xd, Wd, rs)[0] == p0
        assert nv.zkvc_prove_mode(pk, nv.ZKVC_PROVE_CHAIN, Xd, Wd, rs)[0] == p0
    for bad in ([2048, 0, 0, 0, 0, 0, 0, 0, 0, 0], [0, 0, 0, 0, 7, 0, 0, 0, 0, 0], [0, 0, 0, 0, 12, 0, 0, 0, 0, 0],
                [0, 0, 0, 0, 0, 3, 0, 0, 0, 0], [0, 0, 0, 0, 0, 0, 2, 0, 0, 0], [0, 0, 0, 0, 0, 0, 0, 2, 0, 0],
                [0, 0, 0, 0, 0, 0, 0, 0, 2, 0]):
        with pytest.raises(nv.ZkvcError):
            nv.zkvc_pk_set_tuning(pk, bad)


@pytest.mark.parametrize("mode", ["fold", "chain"])
def test_stage_timeline_follows_the_stream_joins(nv, mode):
    """The stage spans of a proof respect the prover's dependencies: the NTTs follow the
    witness, the H-query MSM follows the NTTs, and the encoding of C follows every side
    stream (H, G2 with B's encoding, the small-digit run with what follows it)."""
    import torch
    a, n, b = 5, 7, 3
    inst = inputs.instance(31, (a, n, b))
    pk, _ = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    m = {"fold": nv.ZKVC_PROVE_FOLD, "chain": nv.ZKVC_PROVE_CHAIN}[mode]
    Xd, Wd = torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda()
    rs = inputs.to_bytes32(inst["rs"])
    ref = nv.zkvc_prove_mode(pk, m, Xd, Wd, rs)[0]
    nv.zkvc_profile_enable(True)
    try:
        for _ in range(3):
            assert nv.zkvc_prove_mode(pk, m, Xd, Wd, rs)[0] == ref
        prof = nv.zkvc_profile_read()
    finally:
        nv.zkvc_profile_enable(False)
    span = {k: (v["start_ms"], v["end_ms"]) for k, v in prof.items() if v["calls"]}
    for k in ("witness", "ntt", "msm_g1", "msm_g2", "msm_g1_small", "combine"):
        assert prof[k]["calls"] == 3, k
        assert 0.0 <= span[k][0] <= span[k][1], k
    eps = 1e-3
    assert span["witness"][0] == 0.0
    assert span["ntt"][0] >= span["witness"][1] - eps
    assert span["msm_g1"][0] >= span["ntt"][1] - eps
    for k in ("msm_g1", "msm_g2", "msm_g1_small"):
        assert span["combine"][0] >= span[k][1] - eps, k


def test_graph_replays_match_direct_proofs(nv):
    """zkvc_prove captures the proof as a CUDA graph once the same buffers come back and
    replays it afterwards: every replayed proof (new r, s each time, both modes, a change
    of tuning in between) equals the proof of a direct enqueue with fresh buffers, and a
    replay runs as many kernels as a direct proof."""
    import torch
    a, n, b = 5, 7, 3
    inst = inputs.instance(37, (a, n, b))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    rng = random.Random(38)
    rss = [inputs.to_bytes32((rng.randrange(1, bn.R), rng.randrange(1, bn.R))) for _ in range(10)]

    def direct(mode, rs):  # fresh buffers every call: never the captured ones
        Xd, Wd = torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda()
        return nv.zkvc_prove_mode(pk, mode, Xd, Wd, rs)[0]

    Xd, Wd = torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda()
    Yd = torch.empty((a, b), dtype=torch.int32, device="cuda")
    for mode in (nv.ZKVC_PROVE_CHAIN, nv.ZKVC_PROVE_FOLD):
        ws = torch.empty(nv.zkvc_prove_workspace_bytes_mode(pk, mode), dtype=torch.uint8, device="cuda")
        l0 = nv.zkvc_kernel_launches()
        ref0 = direct(mode, rss[0])
        per_direct = nv.zkvc_kernel_launches() - l0
        for i, rs in enumerate(rss):
            proof = nv.zkvc_prove_mode(pk, mode, Xd, Wd, rs, Y=Yd, workspace=ws)[0]
            assert proof == (ref0 if i == 0 else direct(mode, rs)), (mode, i)
            assert np.array_equal(Yd.cpu().numpy(), inst["X"].astype(np.int64) @ inst["W"].astype(np.int64))
        l1 = nv.zkvc_kernel_launches()
        nv.zkvc_prove_mode(pk, mode, Xd, Wd, rss[3], Y=Yd, workspace=ws)
        assert nv.zkvc_kernel_launches() - l1 == per_direct
    # a new tuning re-arms the capture; proofs stay the same
    t = nv.zkvc_pk_get_tuning(pk)
    t2 = list(t)
    t2[2] = 16 if t[2] != 16 else 32
    nv.zkvc_pk_set_tuning(pk, t2)
    ws = torch.empty(nv.zkvc_prove_workspace_bytes(pk), dtype=torch.uint8, device="cuda")
    mode = t2[6]
    for rs in rss[:4]:
        assert nv.zkvc_prove(pk, Xd, Wd, rs, Y=Yd, workspace=ws)[0] == direct(mode, rs)
    X, W = _mats(inst["X"], inst["W"])
    Y = (inst["X"].astype(np.int64) @ inst["W"].astype(np.int64)).tolist()
    assert nv.zkvc_verify(vk, inst["X"], np.array(Y, dtype=np.int32), nv.zkvc_prove(pk, Xd, Wd, rss[5], Y=Yd,
                                                                                     workspace=ws)[0])
