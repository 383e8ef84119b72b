"""Pins of the oracle's nonlinear gadgets (zkVC Sec. III-C) on the matmul output.

* Max verification: the witness's x_max is the row maximum (ties included); a wrong
  x_max, above the maximum (no factor of prod_j (x_max - x_j) vanishes) or below it
  (some x_max - x_j is negative and has no 32-bit decomposition), leaves a row unsatisfied.
* Exponential: the gadget's output is (1 + x/8)^8 of its input rounded to the division by
  2^3, as an exact fraction; within 7/2^12 of (1 + x/8)^8 at the unrounded x; within 0.04
  of e^x on [-8, 0] (the approximation's own error); 0 below T = -8; 1 at x = 0.
* GELU: the output is x^2/8 + x/4 + 1/2 exactly.
* Both circuits: the honest witness satisfies every row, tampered gadget outputs or a
  tampered Y do not, and the per-entry layout holds the values the definitions give."""
import math
import random
from fractions import Fraction

import pytest

from oracle import bn254 as bn
from oracle import crpc, gadgets

F = gadgets.FRAC_BITS
M = gadgets.EXP_SQUARINGS
SCALE_E = 1 << (F * (1 << M))


def _mats(a, n, b, seed):
    rng = random.Random(seed)
    X = [[rng.randint(-128, 127) for _ in range(n)] for _ in range(a)]
    W = [[rng.randint(-128, 127) for _ in range(b)] for _ in range(n)]
    return X, W


def _softmax_circuit(Y, x_max=None):
    """Rows and witness of the SoftMax gadget alone over a given Y (variables: one, Y, aux)."""
    a, b = len(Y), len(Y[0])
    yvar = lambda i, j: 1 + i * b + j
    aux0 = 1 + a * b
    rows = gadgets.gadget_rows("softmax", a, b, yvar, aux0)
    w = [0] * (aux0 + gadgets.aux_count("softmax", a, b))
    w[0] = 1
    for i in range(a):
        for j in range(b):
            w[yvar(i, j)] = bn.fr_from_int(Y[i][j])
    gadgets.gadget_witness("softmax", Y, w, aux0, x_max)
    return rows, w, aux0


@pytest.mark.parametrize("Y", [[[5]], [[3, 9, -4, 9]], [[-7, -2], [0, 0]], [[100, -100, 50, 99, 100, -5]]])
def test_max_verification(Y):
    rows, w, aux0 = _softmax_circuit(Y)
    assert crpc.unsatisfied_rows(rows, w) == []
    b = len(Y[0])
    for i, row in enumerate(Y):
        assert w[aux0 + i * gadgets.softmax_row_aux(b)] == bn.fr_from_int(max(row))


@pytest.mark.parametrize("Y", [[[3, 9, -4, 9]], [[100, -100, 50, 99, 100, -5]], [[5]], [[1, 2]]])
def test_wrong_max_fails(Y):
    top = [max(r) for r in Y]
    second = [max([v for v in r if v != max(r)], default=max(r) - 1) for r in Y]
    for wrong in ([t + 1 for t in top], [t - 1 for t in top], second):
        rows, w, _ = _softmax_circuit(Y, x_max=wrong)
        assert crpc.unsatisfied_rows(rows, w) != [], wrong


def test_exp_against_closed_forms():
    T = gadgets.EXP_THRESHOLD
    ds = [0, 1, 7, 8, 9, 1 << F, 3 << F, T - 8, T - 1, T, T + 1, 2 * T, (1 << 20) + 5, (1 << 32) - 1]
    ds += random.Random(3).sample(range(T + 1), 40)
    for d in ds:
        c, q, beta, es = gadgets.exp_approx_fixed(d)
        got = Fraction(es[-1], SCALE_E)
        assert es == [beta ** (1 << t) for t in range(1, M + 1)]
        if d > T:
            assert c == 0 and got == 0, d
            continue
        x_rounded = Fraction(-(d >> M) * (1 << M), 1 << F)
        assert got == (1 + x_rounded / (1 << M)) ** (1 << M), d
        x = Fraction(-d, 1 << F)
        assert abs(got - (1 + x / (1 << M)) ** (1 << M)) <= Fraction(7, 1 << F), d
        assert abs(float(got) - math.exp(float(x))) <= 0.04, d
    assert gadgets.exp_approx_fixed(0)[3][-1] == SCALE_E               # e^0 = 1
    assert gadgets.exp_approx_fixed(T)[3][-1] == 0                     # joins the clipped branch


def test_gelu_polynomial():
    for y in [0, 1, -1, 1 << F, -(1 << F), 3 << F, -(5 << F), 12345, -98765, (1 << 24) - 1, -(1 << 24)]:
        x = Fraction(y, 1 << F)
        assert Fraction(gadgets.gelu_fixed(y), 1 << (2 * F + 3)) == x * x / 8 + x / 4 + Fraction(1, 2), y


@pytest.mark.parametrize("circuit", ["crpc_psq_softmax", "crpc_psq_gelu"])
@pytest.mark.parametrize("pub", crpc.PUBLIC_IO)
def test_gadget_circuits_satisfied_and_tamper(circuit, pub):
    z = 0xABCDEF12345 % bn.R
    for a, n, b in [(1, 1, 1), (2, 3, 4), (3, 5, 2)]:
        sh = crpc.Shape(a, n, b, circuit, pub)
        X, W = _mats(a, n, b, 7 * a + n + 13 * b)
        rows = crpc.build_r1cs(sh, z)
        assert len(rows) == sh.n_rows
        w = crpc.witness(sh, X, W, z)
        assert crpc.unsatisfied_rows(rows, w) == []
        Y = crpc.matmul_int(X, W)
        aux0 = sh.gadget_aux0()
        if circuit == "crpc_psq_gelu":
            for i in range(a):
                for j in range(b):
                    assert w[aux0 + i * b + j] == bn.fr_from_int(gadgets.gelu_fixed(Y[i][j]))
            last = aux0 + a * b - 1
        else:
            outs = gadgets.softmax_outputs(Y)
            per = gadgets.softmax_row_aux(b)
            for i in range(a):
                ent0 = aux0 + i * per + 1 + max(0, b - 2)
                for j in range(b):
                    e = ent0 + j * gadgets.SOFTMAX_PER_ENTRY + gadgets.SOFTMAX_PER_ENTRY - 1
                    assert w[e] == outs[i][j] % bn.R
            last = aux0 + a * per - 1                    # the last entry's output
        bad = list(w)
        bad[last] = (bad[last] + 1) % bn.R
        assert crpc.unsatisfied_rows(rows, bad) != []
        Yt = [r[:] for r in Y]
        Yt[0][0] += 1
        assert crpc.unsatisfied_rows(rows, crpc.witness(sh, X, W, z, Yt)) != []
