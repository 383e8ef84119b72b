"""Pins of the oracle's CRPC + PSQ constraint system against the paper's worked example,
its counting claims and negative examples, and integer arithmetic."""
import os
import random

import numpy as np

from oracle import bn254 as bn
from oracle import crpc

R = bn.R
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                out.append(line.split())
    return out


def _rand_mats(a, n, b, seed):
    rng = random.Random(seed)
    X = [[rng.randint(-128, 127) for _ in range(n)] for _ in range(a)]
    W = [[rng.randint(-128, 127) for _ in range(b)] for _ in range(n)]
    return X, W


def test_worked_example_exponents():
    """Sec. III-A: X_0(Z) = x00 + Z^2 x10 + Z^4 x20, W_0(Z) = w00 + Z w01, Y(Z) up to Z^5."""
    g = _read_golden("crpc_worked_example.txt")
    a, n, b = (int(v) for v in g[0][1:])
    sh = crpc.Shape(a, n, b)
    z = 0x1234567890ABCDEF
    rows = crpc.build_r1cs(sh, z, with_input_rows=False)
    for rec in g[1:]:
        if rec[0] == "X":
            i, k, e = map(int, rec[1:])
            assert rows[k][0][sh.x(i, k)] == pow(z, e, R)
        elif rec[0] == "W":
            k, j, e = map(int, rec[1:])
            assert rows[k][1][sh.w(k, j)] == pow(z, e, R)
        elif rec[0] == "Y":
            i, j, e = map(int, rec[1:])
            assert rows[n - 1][2][sh.y(i, j)] == pow(z, e, R)
        elif rec[0] == "constraints_crpc":
            assert len(rows) == int(rec[1])
        elif rec[0] == "constraints_vanilla":
            assert crpc.vanilla_matmul_constraint_count(a, n, b) == int(rec[1])


def _int_poly_mul(p, q):
    out = [0] * (len(p) + len(q) - 1)
    for i, x in enumerate(p):
        for j, y in enumerate(q):
            out[i + j] += x * y
    return out


def test_crpc_identity_as_integer_polynomials():
    """sum_(i,j) Z^(ib+j) y_ij = sum_k X_k(Z) W_k(Z) holds coefficient by coefficient."""
    for (a, n, b) in [(3, 2, 2), (4, 16, 8), (5, 3, 7), (1, 4, 1)]:
        X, W = _rand_mats(a, n, b, a * 100 + n)
        Y = (np.array(X, dtype=np.int64) @ np.array(W, dtype=np.int64)).tolist()
        lhs = [0] * (a * b)
        for i in range(a):
            for j in range(b):
                lhs[i * b + j] = Y[i][j]
        rhs = [0] * (a * b)
        for k in range(n):
            Xk = [0] * ((a - 1) * b + 1)
            for i in range(a):
                Xk[i * b] = X[i][k]
            Wk = [W[k][j] for j in range(b)]
            for e, c in enumerate(_int_poly_mul(Xk, Wk)):
                rhs[e] += c
        assert lhs == rhs


def test_matmul_int_matches_numpy():
    X, W = _rand_mats(6, 9, 5, 3)
    ref = (np.array(X, dtype=np.int64) @ np.array(W, dtype=np.int64)).tolist()
    assert crpc.matmul_int(X, W) == ref


def test_witness_satisfies_r1cs():
    for (a, n, b) in [(4, 16, 8), (3, 2, 2), (2, 1, 3), (1, 5, 1)]:
        sh = crpc.Shape(a, n, b)
        X, W = _rand_mats(a, n, b, n)
        z = random.Random(n).randrange(2, R)
        rows = crpc.build_r1cs(sh, z)
        w = crpc.witness(sh, X, W, z)
        assert crpc.unsatisfied_rows(rows, w) == []
        # the final prefix sum plus the last product is Y(z)  (PSQ closes against Y)
        ak, bk = crpc.crpc_evaluations(X, W, z)
        Y = crpc.matmul_int(X, W)
        assert sum(x * y for x, y in zip(ak, bk)) % R == crpc.crpc_y_at_z(Y, z)


def test_tampered_output_rejected():
    """Soundness statement of Sec. II: a wrong y_ij must not satisfy the constraints."""
    sh = crpc.Shape(4, 16, 8)
    X, W = _rand_mats(4, 16, 8, 11)
    z = 987654321987654321
    rows = crpc.build_r1cs(sh, z)
    Y = crpc.matmul_int(X, W)
    Y[2][5] += 1
    w = crpc.witness(sh, X, W, z, Y)
    assert crpc.unsatisfied_rows(rows, w) == [sh.n - 1]


def test_counts_and_shape_sizes():
    # Sec. III-A: n constraints instead of a b n
    for (a, n, b) in [(4, 16, 8), (49, 320, 512)]:
        sh = crpc.Shape(a, n, b)
        assert sh.n_rows - (sh.n_public + 1) == n
        assert crpc.vanilla_matmul_constraint_count(a, n, b) == a * b * n
    sh = crpc.Shape(4, 16, 8)
    assert (sh.n_public, sh.n_vars, sh.domain) == (96, 240, 128)
    sh = crpc.Shape(49, 320, 512)
    assert (sh.n_public, sh.n_vars, sh.domain) == (40768, 204928, 1 << 16)


def test_psq_left_wires():
    """Sec. III-B: a 3-term dot product needs 4 constraints / 6 left wires without PSQ and
    3 constraints / 3 left wires with it."""
    g = {rec[0]: int(rec[1]) for rec in _read_golden("psq_dot_product.txt")}
    n = g["terms"]
    without = crpc.dot_product_rows_without_psq(n)
    assert len(without) == g["without_psq_constraints"]
    assert crpc.left_wire_count(without) == g["without_psq_left_wires"]
    psq = crpc.build_r1cs(crpc.Shape(1, n, 1), 5, with_input_rows=False)
    assert len(psq) == g["with_psq_constraints"]
    assert crpc.left_wire_count(psq) == g["with_psq_left_wires"]
    # and the PSQ chain computes the dot product: the prefix sums are the running totals
    X = [[3, -4, 7]]
    W = [[2], [5], [-6]]
    w = crpc.witness(crpc.Shape(1, n, 1), X, W, 5)
    sh = crpc.Shape(1, n, 1)
    assert w[sh.s(0)] == 6 and w[sh.s(1)] == (6 - 20) % R


def test_sum_transformation_is_unsound():
    """Sec. III-A: the 'intuitive' sum transformation accepts a Y whose total is right but
    whose entries are not; CRPC at a random z rejects it."""
    X, W = _rand_mats(3, 2, 2, 21)
    Y = crpc.matmul_int(X, W)
    Yt = [row[:] for row in Y]
    Yt[0][0] += 5
    Yt[1][1] -= 5
    total = sum(sum(r) for r in Yt)
    rhs = sum(sum(X[i][k] for i in range(3)) * sum(W[k][j] for j in range(2)) for k in range(2))
    assert total == rhs and Yt != Y
    sh = crpc.Shape(3, 2, 2)
    z = 31337
    rows = crpc.build_r1cs(sh, z)
    assert crpc.unsatisfied_rows(rows, crpc.witness(sh, X, W, z, Yt)) != []


def test_dummy_term_transformation_is_not_an_identity():
    """Sec. III-A: the interleaved-power (vCNN-style) product is not equal to the Y
    polynomial; its Z^1 coefficient is y00 but superfluous cross terms remain."""
    X, W = _rand_mats(3, 2, 2, 22)
    Y = crpc.matmul_int(X, W)
    lhs = [0] * 12
    for (i, j), e in {(0, 0): 1, (0, 1): 3, (1, 0): 5, (1, 1): 7, (2, 0): 9, (2, 1): 11}.items():
        lhs[e] = Y[i][j]
    xpoly = [0] * 10
    for (i, k), e in {(0, 0): 1, (0, 1): 0, (1, 0): 5, (1, 1): 4, (2, 0): 9, (2, 1): 8}.items():
        xpoly[e] += X[i][k]
    wpoly = [0] * 4
    for (k, j), e in {(0, 0): 0, (0, 1): 2, (1, 0): 1, (1, 1): 3}.items():
        wpoly[e] += W[k][j]
    rhs = _int_poly_mul(xpoly, wpoly)
    lhs += [0] * (len(rhs) - len(lhs))
    assert rhs != lhs
    assert rhs[1] == Y[0][0]
