"""Pins of the oracle's circuit variants (the Sec. V / Table II ablation: CRPC with and
without PSQ, PSQ without CRPC, vanilla) and of the private-input mode: the true witness
satisfies every row; a tampered output breaks some row; the row, variable and left-wire
counts follow from the definitions (vanilla: a b n product rows, Sec. III-A; PSQ halves
the left wires of a dot product, Sec. III-B); Groth16 over each circuit proves and
verifies, the closed-form proof equals the naive one, and a wrong statement fails."""
import itertools
import random

import pytest

from oracle import bn254 as bn
from oracle import crpc, groth16 as og

SHAPES = [(1, 1, 1), (2, 3, 2), (3, 2, 4)]
COMBOS = list(itertools.product(crpc.CIRCUITS, crpc.PUBLIC_IO))


def _mats(a, n, b, seed):
    rng = random.Random(seed)
    X = [[rng.randint(-128, 127) for _ in range(n)] for _ in range(a)]
    W = [[rng.randint(-128, 127) for _ in range(b)] for _ in range(n)]
    return X, W


@pytest.mark.parametrize("circuit,pub", COMBOS)
def test_satisfaction_and_counts(circuit, pub):
    z = 0x1234567 * 7919 % bn.R
    for a, n, b in SHAPES:
        sh = crpc.Shape(a, n, b, circuit, pub)
        X, W = _mats(a, n, b, a * 100 + n * 10 + b)
        rows = crpc.build_r1cs(sh, z)
        assert len(rows) == sh.n_rows
        # gadget rows (Sec. III-C): per SoftMax entry 32 + 1 bit/recomposition rows for d,
        # 33 + 1 for u, the base and 3 squarings; a product chain of max(1, b - 1) rows per
        # row of Y; one GELU row per entry
        circuit_rows = {"crpc_psq": n, "crpc": n + 1, "psq": a * b * n, "vanilla": a * b * n + a * b,
                        "crpc_psq_softmax": n + a * (b * 71 + max(1, b - 1)),
                        "crpc_psq_gelu": n + a * b}[circuit]
        assert sh.n_rows == circuit_rows + (a * n + a * b if pub == "xy" else 0) + 1
        w = crpc.witness(sh, X, W, z)
        assert len(w) == sh.n_vars
        assert crpc.unsatisfied_rows(rows, w) == []
        Y = crpc.matmul_int(X, W)
        Y[0][0] += 1
        bad = crpc.witness(sh, X, W, z, Y)
        assert crpc.unsatisfied_rows(rows, bad) != []
        # every variable index is used exactly once by the layout
        used = set()
        for i in range(a):
            for k in range(n):
                used.add(sh.x(i, k))
            for j in range(b):
                used.add(sh.y(i, j))
        for k in range(n):
            for j in range(b):
                used.add(sh.w(k, j))
        used |= {sh.aux(t) for t in range(sh.n_aux)}
        assert used == set(range(1, sh.n_vars))


def test_left_wires_halved_by_psq():
    """Left wires (A entries) of the circuit rows: vanilla 2 a b n, PSQ-only a b n
    (Sec. III-B: PSQ removes the summing row's long combination); CRPC n a + n versus
    CRPC + PSQ n a."""
    a, n, b = 2, 5, 3
    lw = {}
    for c in crpc.CIRCUITS:
        sh = crpc.Shape(a, n, b, c)
        lw[c] = crpc.left_wire_count(crpc.build_r1cs(sh, 3, with_input_rows=False))
    assert lw["vanilla"] == 2 * a * b * n and lw["psq"] == a * b * n
    assert lw["crpc"] == n * a + n and lw["crpc_psq"] == n * a
    assert crpc.Shape(a, n, b, "vanilla").n_circuit_rows - a * b == crpc.vanilla_matmul_constraint_count(a, n, b)


@pytest.mark.parametrize("circuit,pub", COMBOS)
def test_groth16_over_each_circuit(circuit, pub):
    a, n, b = 2, 3, 2
    sh = crpc.Shape(a, n, b, circuit, pub)
    rng = random.Random(10 * crpc.CIRCUITS.index(circuit) + crpc.PUBLIC_IO.index(pub))
    toxic = [rng.randrange(2, bn.R) for _ in range(6)]
    X, W = _mats(a, n, b, 42)
    pk, vk = og.setup(sh, toxic)
    assert len(vk.IC) == sh.n_public + 1
    r, s = rng.randrange(bn.R), rng.randrange(bn.R)
    proof, Y, h = og.prove(pk, X, W, r, s)
    assert h[sh.domain - 1] == 0
    cf, _ = og.closed_form_proof(sh, toxic, X, W, r, s)
    assert og.proof_bytes(cf) == og.proof_bytes(proof)
    assert og.verify(vk, X, Y, proof)
    bad = dict(proof)
    bad["C"] = bn.g1_add(proof["C"], bn.G1_GEN)
    assert not og.verify(vk, X, Y, bad)
    if pub == "xy":
        Yt = [row[:] for row in Y]
        Yt[1][1] += 1
        assert not og.verify(vk, X, Yt, proof)
