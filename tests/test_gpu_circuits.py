"""GPU parity of the generic sparse-R1CS prover over the ablation circuits (Sec. V,
Table II: CRPC + PSQ, CRPC without PSQ, PSQ without CRPC, vanilla), the nonlinear gadget
circuits of Sec. III-C (SoftMax's max verification and exponential, GELU, on the matmul
output) and the private-input mode: every key entry, verifying-key entry and proof equals the oracle's byte for byte on
small shapes; the generic CRPC + PSQ key proves the same bytes as the specialised prover;
at the full [49,320] x [320,512] size every circuit's proof verifies under the library's
pairing verifier and a perturbed one does not."""
import itertools

import numpy as np
import pytest

from oracle import bn254 as bn
from oracle import crpc, groth16 as og
from paper_2504_12217_gb300 import inputs
from tests import _util

pytestmark = pytest.mark.gpu

COMBOS = list(itertools.product(crpc.CIRCUITS, crpc.PUBLIC_IO))
SHAPES = [(1, 1, 1), (2, 3, 2), (3, 5, 4)]
# the Sec. III-C gadget circuits: rows of Y with one entry (the product chain's b = 1
# row), two (no product variable) and five; 71 rows per entry keep the oracle's setup short
GADGET_SHAPES = [(1, 1, 1), (2, 2, 2), (2, 3, 5)]


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _by_var(pk_list, var_list, n_vars, enc, width):
    out = [bytes(width)] * n_vars
    for v, p in zip(var_list, pk_list):
        out[v] = enc(p)
    return b"".join(out)


@pytest.mark.parametrize("circuit,pub", COMBOS)
def test_keys_and_proofs_match_oracle(nv, circuit, pub):
    import torch
    for si, (a, n, b) in enumerate(GADGET_SHAPES if crpc.gadget_of(circuit) else SHAPES):
        seed = 9000 + 100 * crpc.CIRCUITS.index(circuit) + 10 * crpc.PUBLIC_IO.index(pub) + si
        toxic = inputs.setup_values(seed)
        sh = crpc.Shape(a, n, b, circuit, pub)
        pk, vk = nv.zkvc_setup_circuit(a, n, b, circuit, pub, inputs.to_bytes32(toxic))
        info = nv.zkvc_pk_circuit(pk)
        assert (info["rows"], info["vars"]) == (sh.n_rows, sh.n_vars)
        assert pk.log_domain == sh.domain.bit_length() - 1
        opk, ovk = og.setup(sh, toxic)
        V = sh.n_vars
        assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_A, 0, V) == _by_var(opk.A, opk.A_vars, V, bn.g1_bytes, 64)
        assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_B1, 0, V) == _by_var(opk.B1, opk.B_vars, V, bn.g1_bytes, 64)
        assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_B2, 0, V) == _by_var(opk.B2, opk.B_vars, V, bn.g2_bytes, 128)
        assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_L, 0, V) == _by_var(opk.L, opk.L_vars, V, bn.g1_bytes, 64)
        assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_H, 0, len(opk.H)) == b"".join(bn.g1_bytes(p) for p in opk.H)
        assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_DELTA1, 0, 1) == bn.g1_bytes(opk.delta1)
        assert nv.zkvc_pk_export(pk, nv.ZKVC_Q_DELTA2, 0, 1) == bn.g2_bytes(opk.delta2)
        assert nv.zkvc_vk_export(vk, nv.ZKVC_VK_IC, 0, len(ovk.IC)) == b"".join(bn.g1_bytes(p) for p in ovk.IC)
        assert nv.zkvc_vk_export(vk, nv.ZKVC_VK_GAMMA2, 0, 1) == bn.g2_bytes(ovk.gamma2)
        X, W = inputs.matrices(seed, a, n, b)
        for rs in (inputs.prover_values(seed), [0, 1]):
            proof, Y = nv.zkvc_prove(pk, torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(), inputs.to_bytes32(rs))
            oproof, oY, _ = og.prove(opk, X.astype(int).tolist(), W.astype(int).tolist(), *rs)
            assert Y.cpu().numpy().tolist() == oY
            assert proof == og.proof_bytes(oproof), (circuit, pub, (a, n, b), rs)
            Xv, Yv = (X, Y.cpu().numpy()) if pub == "xy" else (None, None)
            assert nv.zkvc_verify(vk, Xv, Yv, proof)


def test_generic_crpc_psq_equals_specialised(nv):
    """The same circuit and toxic waste through both provers give identical proofs."""
    import torch
    for (a, n, b) in ((4, 16, 8), (5, 40, 33)):
        toxic = inputs.setup_values(77 + a)
        pk_s, _ = nv.zkvc_setup(a, n, b, inputs.to_bytes32(toxic))
        pk_g, vk_g = nv.zkvc_setup_circuit(a, n, b, "crpc_psq", "xy", inputs.to_bytes32(toxic))
        X, W = inputs.matrices(78 + a, a, n, b)
        rs = inputs.to_bytes32(inputs.prover_values(79 + a))
        Xd, Wd = torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda()
        p_s, _ = nv.zkvc_prove(pk_s, Xd, Wd, rs)
        p_g, Y = nv.zkvc_prove(pk_g, Xd, Wd, rs)
        assert p_s == p_g
        assert nv.zkvc_verify(vk_g, X, Y.cpu().numpy(), p_g)


def test_generic_keys_are_rejected_where_unsupported(nv, tmp_path):
    toxic = inputs.setup_values(5)
    pk, _ = nv.zkvc_setup_circuit(2, 3, 2, "vanilla", "xy", inputs.to_bytes32(toxic))
    with pytest.raises(nv.ZkvcError):
        nv.zkvc_pk_save(pk, str(tmp_path / "k.pk"))
    with pytest.raises(nv.ZkvcError):
        nv.Batch([pk])
    with pytest.raises(nv.ZkvcError):
        nv.Server([pk], slots=1, mem_budget=1 << 24)
    with pytest.raises(nv.ZkvcError):
        nv.zkvc_setup_circuit(2, 3, 2, 7, 0, inputs.to_bytes32(toxic))


@pytest.mark.parametrize("circuit", list(crpc.CIRCUITS))
def test_full_size_every_circuit_verifies(nv, circuit):
    """[49,320] x [320,512] (vanilla: 8.05 M rows, N = 2^23): each circuit's GPU proof
    verifies under the pairing verifier (X and Y public), a perturbed C does not, and Y is
    the integer product."""
    import torch
    a, n, b = inputs.SHAPE_CFG2
    inst = inputs.instance(inputs.SEED_CFG[2], (a, n, b))
    pk, vk = nv.zkvc_setup_circuit(a, n, b, circuit, "xy", inputs.to_bytes32(inst["toxic"]))
    proof, Y = nv.zkvc_prove(pk, torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda(),
                             inputs.to_bytes32(inst["rs"]))
    Yh = Y.cpu().numpy()
    assert np.array_equal(Yh, inst["X"].astype(np.int64) @ inst["W"].astype(np.int64))
    assert nv.zkvc_verify(vk, inst["X"], Yh, proof)
    bad = proof[:192] + bn.g1_bytes(bn.g1_add(bn.g1_from_bytes(proof[192:]), bn.G1_GEN))
    assert not nv.zkvc_verify(vk, inst["X"], Yh, bad)
    if circuit == "crpc_psq":
        cf, _ = og.closed_form_proof(crpc.Shape(a, n, b), inst["toxic"], inst["X"].astype(int).tolist(),
                                     inst["W"].astype(int).tolist(), *inst["rs"])
        assert proof == og.proof_bytes(cf)


def test_full_size_private_io(nv):
    """X and Y private at [49,320] x [320,512]: N = 2^9, the proof verifies without inputs."""
    import torch
    a, n, b = inputs.SHAPE_CFG2
    inst = inputs.instance(inputs.SEED_CFG[2], (a, n, b))
    pk, vk = nv.zkvc_setup_circuit(a, n, b, "crpc_psq", "none", inputs.to_bytes32(inst["toxic"]))
    assert pk.log_domain == 9
    proof, Y = nv.zkvc_prove(pk, torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda(),
                             inputs.to_bytes32(inst["rs"]))
    assert nv.zkvc_verify(vk, None, None, proof)
    cf, _ = og.closed_form_proof(crpc.Shape(a, n, b, "crpc_psq", "none"), inst["toxic"], inst["X"].astype(int).tolist(),
                                 inst["W"].astype(int).tolist(), *inst["rs"])
    assert proof == og.proof_bytes(cf)
