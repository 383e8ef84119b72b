"""Pins of the oracle's QAP and Groth16: Lagrange basis, the quotient identity, honest
proofs verify, tampered ones do not, and the naive proof equals the closed form."""
import random

import pytest

from oracle import bn254 as bn
from oracle import crpc, groth16 as g
from oracle import ntt as nt

R = bn.R


def _rand_mats(a, n, b, seed):
    rng = random.Random(seed)
    X = [[rng.randint(-128, 127) for _ in range(n)] for _ in range(a)]
    W = [[rng.randint(-128, 127) for _ in range(b)] for _ in range(n)]
    return X, W


def test_lagrange_closed_form():
    tau = 0xDEADBEEF12345
    for N in (4, 16):
        Lk = g.lagrange_at(tau, N)
        for k in range(N):
            assert Lk[k] == g.lagrange_at_product(tau, N, k)
        # interpolation: sum_k L_k(tau) f(omega^k) = f(tau) for deg f < N
        coeffs = [random.Random(N).randrange(R) for _ in range(N)]
        ev = nt.ntt(coeffs)
        assert sum(l * v for l, v in zip(Lk, ev)) % R == nt.poly_eval(coeffs, tau)


def test_quotient_identity():
    sh = crpc.Shape(4, 16, 8)
    X, W = _rand_mats(4, 16, 8, 1)
    z = 555
    rows = crpc.build_r1cs(sh, z)
    w = crpc.witness(sh, X, W, z)
    N = sh.domain
    Aev, Bev, Cev = g.domain_evaluations(rows, w, N)
    h, (a, b, c) = g.quotient(Aev, Bev, Cev)
    assert h[N - 1] == 0
    omega = bn.fr_root_of_unity(N)
    for k in (0, 1, 77):                         # coefficients interpolate the evaluations
        x = pow(omega, k, R)
        assert nt.poly_eval(a, x) == Aev[k] and nt.poly_eval(c, x) == Cev[k]
    zeta = 0xABCDEF0123456789
    t = (pow(zeta, N, R) - 1) % R
    lhs = nt.poly_eval(h, zeta) * t % R
    rhs = (nt.poly_eval(a, zeta) * nt.poly_eval(b, zeta) - nt.poly_eval(c, zeta)) % R
    assert lhs == rhs


def test_quotient_detects_unsatisfied_witness():
    sh = crpc.Shape(2, 3, 2)
    X, W = _rand_mats(2, 3, 2, 2)
    z = 777
    rows = crpc.build_r1cs(sh, z)
    Y = crpc.matmul_int(X, W)
    Y[1][1] += 1
    w = crpc.witness(sh, X, W, z, Y)
    Aev, Bev, Cev = g.domain_evaluations(rows, w, sh.domain)
    h, _ = g.quotient(Aev, Bev, Cev)
    assert h[sh.domain - 1] != 0


@pytest.fixture(scope="module")
def cfg1_keys():
    sh = crpc.Shape(4, 16, 8)
    rng = random.Random(42)
    toxic = [rng.randrange(1, R) for _ in range(6)]
    pk, vk = g.setup(sh, toxic)
    X, W = _rand_mats(4, 16, 8, 42)
    return sh, toxic, pk, vk, X, W


def test_honest_proof_verifies_and_matches_closed_form(cfg1_keys):
    sh, toxic, pk, vk, X, W = cfg1_keys
    r, s = 0x1111, R - 0x2222
    proof, Y, _ = g.prove(pk, X, W, r, s)
    assert g.verify(vk, X, Y, proof)
    cf, _ = g.closed_form_proof(sh, toxic, X, W, r, s)
    assert g.proof_bytes(cf) == g.proof_bytes(proof)
    assert len(g.proof_bytes(proof)) == 256


def test_tampered_statements_rejected(cfg1_keys):
    sh, toxic, pk, vk, X, W = cfg1_keys
    proof, Y, _ = g.prove(pk, X, W, 3, 4)
    Yt = [row[:] for row in Y]
    Yt[3][7] -= 1
    assert not g.verify(vk, X, Yt, proof)                       # flipped y_ij
    bad = dict(proof)
    bad["A"] = bn.g1_add(proof["A"], bn.G1_GEN)
    assert not g.verify(vk, X, Y, bad)                          # perturbed A
    swapped = {"A": proof["C"], "B": proof["B"], "C": proof["A"]}
    assert not g.verify(vk, X, Y, swapped)                      # swapped A / C


def test_pk_entry_scalars(cfg1_keys):
    sh, toxic, pk, vk, X, W = cfg1_keys
    for q, lst in (("A", pk.A), ("B", pk.B1), ("L", pk.L), ("H", pk.H), ("IC", vk.IC)):
        idx = [0, len(lst) // 2, len(lst) - 1]
        for i, s in zip(idx, g.pk_entry_scalars(sh, toxic, q, idx)):
            assert bn.g1_mul(bn.G1_GEN, s) == lst[i]
    assert len(pk.A) == sh.n_public + 1
    assert len(pk.B1) == sh.n * sh.b and len(pk.L) == sh.n * sh.b + sh.n - 1
    assert len(pk.H) == sh.domain - 1


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 3), (1, 5, 1), (3, 2, 2)])
def test_degenerate_shapes(shape):
    a, n, b = shape
    sh = crpc.Shape(a, n, b)
    rng = random.Random(a * 31 + n * 7 + b)
    toxic = [rng.randrange(1, R) for _ in range(6)]
    pk, vk = g.setup(sh, toxic)
    X, W = _rand_mats(a, n, b, 5)
    r, s = rng.randrange(R), rng.randrange(R)
    proof, Y, _ = g.prove(pk, X, W, r, s)
    assert g.verify(vk, X, Y, proof)
    cf, _ = g.closed_form_proof(sh, toxic, X, W, r, s)
    assert g.proof_bytes(cf) == g.proof_bytes(proof)


def test_zero_randomness_proof_matches_closed_form():
    sh = crpc.Shape(2, 3, 2)
    rng = random.Random(99)
    toxic = [rng.randrange(1, R) for _ in range(6)]
    pk, vk = g.setup(sh, toxic)
    X, W = _rand_mats(2, 3, 2, 6)
    for (r, s) in ((0, 0), (1, 0), (0, R - 1)):
        proof, Y, _ = g.prove(pk, X, W, r, s)
        cf, _ = g.closed_form_proof(sh, toxic, X, W, r, s)
        assert g.proof_bytes(proof) == g.proof_bytes(cf)
