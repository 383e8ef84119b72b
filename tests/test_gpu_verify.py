"""GPU pairing and batched GPU verification.

The GPU pairing e(P, Q) equals the oracle's optimal ate pairing value (its Fp12 = Fp[w]/
(w^12 - 18 w^6 + 82)) after the change of basis from the GPU tower (Fp6[w]/(w^2 - v),
Fp6 = Fp2[v]/(v^3 - xi), so v = w^2 and i = w^6 - 9); it is bilinear and maps infinity to
one.  Batched GPU verification agrees with the host verifier on honest proofs, tampered
statements, perturbed and malformed proofs and a twist point outside the order-r subgroup,
for keys with and without public inputs, and at the full [49,320] x [320,512] size."""
import random

import numpy as np
import pytest

from oracle import bn254 as bn
from oracle import crpc
from oracle import pairing as opair
from paper_2504_12217_gb300 import inputs
from tests import _util


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _tower_to_w(raw):
    """384 bytes of GPU output -> the oracle's 12 coefficients in the w basis."""
    vals = [int.from_bytes(raw[32 * k: 32 * k + 32], "little") for k in range(12)]
    # tower order: (c0.c0, c0.c1, c0.c2, c1.c0, c1.c1, c1.c2) = w^(0, 2, 4, 1, 3, 5)
    ms = [0, 2, 4, 1, 3, 5]
    out = [0] * 12
    for j, m in enumerate(ms):
        a, b = vals[2 * j], vals[2 * j + 1]
        out[m] = (out[m] + a - 9 * b) % bn.P
        out[m + 6] = (out[m + 6] + b) % bn.P
    return tuple(out)


pytestmark = pytest.mark.gpu


def _gpu_pairs(nv, Ps, Qs):
    P = _util.to_cuda(_util.g1_rows(Ps))
    Q = _util.to_cuda(_util.g2_rows(Qs))
    out = nv.zkvc_pairing(P, Q).cpu().numpy()
    return [_tower_to_w(bytes(out[i])) for i in range(len(Ps))]


def test_pairing_equals_oracle(nv):
    rng = random.Random(21)
    Ps = [bn.G1_GEN, bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R)), bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R))]
    Qs = [bn.G2_GEN, bn.G2_GEN, bn.g2_mul(bn.G2_GEN, rng.randrange(1, bn.R))]
    got = _gpu_pairs(nv, Ps, Qs)
    for g, Pt, Q in zip(got, Ps, Qs):
        assert g == opair.pairing(Pt, Q)


def test_pairing_bilinear_and_degenerate(nv):
    rng = random.Random(22)
    a, b = rng.randrange(2, bn.R), rng.randrange(2, bn.R)
    P, Q = bn.g1_mul(bn.G1_GEN, 7), bn.g2_mul(bn.G2_GEN, 11)
    Ps = [bn.g1_mul(P, a), bn.g1_mul(P, a * b % bn.R), P, None, P]
    Qs = [bn.g2_mul(Q, b), Q, bn.g2_mul(Q, a * b % bn.R), Q, None]
    g = _gpu_pairs(nv, Ps, Qs)
    assert g[0] == g[1] == g[2]
    assert g[3] == opair.F12_ONE and g[4] == opair.F12_ONE
    assert g[0] != opair.F12_ONE


def _small_cases(nv):
    """(vk, X, Y, proof, expected) over keys with and without public inputs."""
    import torch
    cases = []
    for shape, circuit, pub in (((2, 3, 2), "crpc_psq", "xy"), ((3, 5, 4), "vanilla", "xy"),
                                ((2, 3, 2), "crpc_psq", "none"), ((4, 16, 8), "crpc", "none")):
        seed = 600 + shape[0] * 10 + crpc.CIRCUITS.index(circuit)
        toxic = inputs.setup_values(seed)
        pk, vk = nv.zkvc_setup_circuit(*shape, circuit, pub, inputs.to_bytes32(toxic))
        X, W = inputs.matrices(seed, *shape)
        proof, Y = nv.zkvc_prove(pk, torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(),
                                 inputs.to_bytes32(inputs.prover_values(seed)))
        Yh = Y.cpu().numpy()
        xs = (X, Yh) if pub == "xy" else (None, None)
        cases.append((vk, xs[0], xs[1], proof, True))
        bad_c = proof[:192] + bn.g1_bytes(bn.g1_add(bn.g1_from_bytes(proof[192:]), bn.G1_GEN))
        cases.append((vk, xs[0], xs[1], bad_c, False))
        cases.append((vk, xs[0], xs[1], proof[192:256] + proof[64:192] + proof[:64], False))
        cases.append((vk, xs[0], xs[1], bytes(256), False))
        cases.append((vk, xs[0], xs[1], bn.P.to_bytes(32, "little") + proof[32:], False))
        if pub == "xy":
            Yt = Yh.copy()
            Yt[0, 0] += 1
            cases.append((vk, X, Yt, proof, False))
    return cases


def _twist_point_off_subgroup():
    rng = random.Random(9)
    P = bn.P
    while True:
        x = (rng.randrange(P), rng.randrange(P))
        rhs = bn.f2_add(bn.f2_mul(bn.f2_mul(x, x), x), bn.B2)
        a, b = rhs
        norm = (a * a + b * b) % P
        n = pow(norm, (P + 1) // 4, P)
        if n * n % P != norm:
            continue
        inv2 = pow(2, -1, P)
        for cand in ((a + n) * inv2 % P, (a - n) * inv2 % P):
            c = pow(cand, (P + 1) // 4, P)
            if c * c % P == cand and c != 0:
                d = b * pow(2 * c, -1, P) % P
                if bn.f2_mul((c, d), (c, d)) == (a % P, b % P):
                    return (x, (c, d))


def test_batch_verify_matches_host(nv):
    cases = _small_cases(nv)
    vk0, X0, Y0, proof0, _ = cases[0]
    Q = _twist_point_off_subgroup()
    assert bn.g2_on_curve(Q) and bn.g2_mul_noshortcut(Q, bn.R) is not None
    cases.append((vk0, X0, Y0, proof0[:64] + bn.g2_bytes(Q) + proof0[192:], False))
    vks = [c[0] for c in cases]
    got = nv.zkvc_verify_batch(vks, [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases])
    assert got == [c[4] for c in cases]
    host = [nv.zkvc_verify(c[0], c[1], c[2], c[3]) for c in cases]
    assert got == host
    assert nv.zkvc_verify_batch([], [], [], []) == []


def test_batch_verify_full_size(nv):
    """[49,320] x [320,512]: the GPU accepts the proof and rejects a perturbed one."""
    import torch
    a, n, b = inputs.SHAPE_CFG2
    inst = inputs.instance(inputs.SEED_CFG[2], (a, n, b))
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    proof, Y = nv.zkvc_prove(pk, torch.from_numpy(inst["X"]).cuda(), torch.from_numpy(inst["W"]).cuda(),
                             inputs.to_bytes32(inst["rs"]))
    Yh = Y.cpu().numpy()
    bad = proof[:192] + bn.g1_bytes(bn.g1_add(bn.g1_from_bytes(proof[192:]), bn.G1_GEN))
    got = nv.zkvc_verify_batch([vk] * 3, [inst["X"]] * 3, [Yh, Yh, Yh + np.int32(1)], [proof, bad, proof])
    assert got == [True, False, False]
