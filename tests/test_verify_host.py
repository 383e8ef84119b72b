"""The library's host verifier (C++ optimal-ate pairing) against oracle-made keys and
proofs: honest proofs verify; tampered statements, perturbed or malformed proofs and a
twist point outside the order-r subgroup do not.  Needs no GPU."""
import random

import numpy as np
import pytest

from oracle import bn254 as bn
from oracle import crpc, groth16 as og
from tests import _util


@pytest.fixture(scope="module")
def setup1():
    nv = _util.native()
    a, n, b = 3, 5, 4
    rng = random.Random(314)
    toxic = [rng.randrange(2, bn.R) for _ in range(6)]
    sh = crpc.Shape(a, n, b)
    opk, ovk = og.setup(sh, toxic)
    X = np.array([[rng.randint(-128, 127) for _ in range(n)] for _ in range(a)], dtype=np.int8)
    W = np.array([[rng.randint(-128, 127) for _ in range(b)] for _ in range(n)], dtype=np.int8)
    proof, Y, _ = og.prove(opk, X.astype(int).tolist(), W.astype(int).tolist(), rng.randrange(bn.R),
                           rng.randrange(bn.R))
    vk = nv.zkvc_vk_import(a, n, b, bn.g1_bytes(ovk.alpha1), bn.g2_bytes(ovk.beta2), bn.g2_bytes(ovk.gamma2),
                           bn.g2_bytes(ovk.delta2), b"".join(bn.g1_bytes(p) for p in ovk.IC))
    return nv, vk, X, np.array(Y, dtype=np.int32), og.proof_bytes(proof)


def test_honest_proof_verifies(setup1):
    nv, vk, X, Y, proof = setup1
    assert nv.zkvc_verify(vk, X, Y, proof)


def test_tampered_statement(setup1):
    nv, vk, X, Y, proof = setup1
    Yt = Y.copy()
    Yt[1, 2] += 1
    assert not nv.zkvc_verify(vk, X, Yt, proof)
    Xt = X.copy()
    Xt[0, 0] = -Xt[0, 0] if Xt[0, 0] not in (0, -128) else 5
    assert not nv.zkvc_verify(vk, Xt, Y, proof)


def test_perturbed_and_malformed_proofs(setup1):
    nv, vk, X, Y, proof = setup1
    A = bn.g1_from_bytes(proof[:64])
    bad = bn.g1_bytes(bn.g1_add(A, bn.G1_GEN)) + proof[64:]
    assert not nv.zkvc_verify(vk, X, Y, bad)
    swapped = proof[192:256] + proof[64:192] + proof[:64]
    assert not nv.zkvc_verify(vk, X, Y, swapped)
    off_curve = proof[:32] + (int.from_bytes(proof[32:64], "little") ^ 1).to_bytes(32, "little") + proof[64:]
    assert not nv.zkvc_verify(vk, X, Y, off_curve)
    non_canonical = bn.P.to_bytes(32, "little") + proof[32:]
    assert not nv.zkvc_verify(vk, X, Y, non_canonical)
    assert not nv.zkvc_verify(vk, X, Y, bytes(256))


def _fp2_sqrt(alpha):
    """Square root in Fp2 (p = 3 mod 4), or None."""
    P = bn.P
    a, b = alpha
    norm = (a * a + b * b) % P
    n = pow(norm, (P + 1) // 4, P)
    if n * n % P != norm:
        return None
    inv2 = pow(2, -1, P)
    for cand in ((a + n) * inv2 % P, (a - n) * inv2 % P):
        c = pow(cand, (P + 1) // 4, P)
        if c * c % P == cand and c != 0:
            d = b * pow(2 * c, -1, P) % P
            if bn.f2_mul((c, d), (c, d)) == (a % P, b % P):
                return (c, d)
    return None


def test_twist_point_outside_subgroup(setup1):
    nv, vk, X, Y, proof = setup1
    rng = random.Random(9)
    while True:
        x = (rng.randrange(bn.P), rng.randrange(bn.P))
        rhs = bn.f2_add(bn.f2_mul(bn.f2_mul(x, x), x), bn.B2)
        y = _fp2_sqrt(rhs)
        if y is not None:
            break
    Q = (x, y)
    assert bn.g2_on_curve(Q) and bn.g2_mul_noshortcut(Q, bn.R) is not None
    bad = proof[:64] + bn.g2_bytes(Q) + proof[192:]
    assert not nv.zkvc_verify(vk, X, Y, bad)


def test_import_rejects_wrong_ic_count():
    nv = _util.native()
    with pytest.raises(nv.ZkvcError):
        nv.zkvc_vk_import(2, 2, 2, bytes(64), bytes(128), bytes(128), bytes(128), bytes(64 * 3))


def test_vk_save_load_round_trip(setup1, tmp_path):
    nv, vk, X, Y, proof = setup1
    path = tmp_path / "key.vk"
    nv.zkvc_vk_save(vk, str(path))
    vk2 = nv.zkvc_vk_load(str(path))
    assert vk2.shape == vk.shape
    assert nv.zkvc_verify(vk2, X, Y, proof)
    for q, cnt in ((nv.ZKVC_VK_IC, 3 * 5 + 3 * 4 + 1), (nv.ZKVC_VK_DELTA2, 1)):
        assert nv.zkvc_vk_export(vk2, q, 0, cnt) == nv.zkvc_vk_export(vk, q, 0, cnt)
    raw = bytearray(path.read_bytes())
    raw[100] ^= 0x40                                # corrupt the payload
    bad = tmp_path / "bad.vk"
    bad.write_bytes(bytes(raw))
    with pytest.raises(nv.ZkvcError) as e:
        nv.zkvc_vk_load(str(bad))
    assert e.value.code == nv.ZKVC_EIO
    short = tmp_path / "short.vk"
    short.write_bytes(path.read_bytes()[:200])      # truncated
    with pytest.raises(nv.ZkvcError):
        nv.zkvc_vk_load(str(short))
    with pytest.raises(nv.ZkvcError):
        nv.zkvc_vk_load(str(tmp_path / "missing.vk"))
