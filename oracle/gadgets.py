"""Nonlinear-function gadgets of zkVC Sec. III-C as rank-1 constraints, on the matmul output.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What the paper states (Sec. III-C, "Nonlinear-Function Approximation"):

* SoftMax over a vector x is computed as e^(x_j - x_max) / sum_j e^(x_j - x_max).
  x_max is verified by two statements: x_max >= x_j for every j (a comparison, done in
  circuits by bit decomposition), and prod_j (x_max - x_j) = 0 (x_max is one of the x_j).
* On the normalised, non-positive inputs x = x_j - x_max, e^x is approximated by 0 below a
  threshold T and by (1 + x/2^n)^(2^n) on [T, 0]; bit decompositions compare x with T and
  divide by 2^n, and the power 2^n is a chain of multiplications.
* GELU(x) is approximated by the polynomial x^2/8 + x/4 + 1/2.

Readings taken here (the paper gives neither the number format, n, T, nor the layout):

* Inputs are the matmul output Y of the CRPC + PSQ circuit (a Transformer layer's scores
  or pre-activations), read as fixed point with F = 12 fractional bits: y stands for
  y / 2^12.  SoftMax runs over each row of Y (b entries), GELU over every entry.
* Exponential: n = 3 (eight-fold power), T = -2^(F + n) / 2^F = -8: exactly where
  1 + x/2^n reaches 0, so the clipped branch joins the polynomial continuously.
* The division by 2^n rounds toward zero on d = x_max - x_j >= 0: q = floor(d / 2^n), and
  the base is 2^F - q (1 + x/2^n at scale 2^F).  The power chain squares without
  rescaling, so e^x is represented exactly as base^(2^n) at scale 2^(F 2^n) (96 bits).
* Bit decompositions: d_j into 32 bits proves x_max >= x_j (|y| < 2^31, so d < 2^32);
  its bits from n up are q, so the division reuses them rather than decomposing d again.
  The threshold comparison decomposes u_j = |T| - d_j + 2^32 into 33 bits; its top bit is
  c_j = [d_j <= |T|].  Each bit b has the row b * b = b, each decomposition one row
  (sum_k 2^k b_k - value) * 1 = 0.
* Clipping multiplies the base by c_j: beta_j = c_j (2^F - q_j); then e_1 = beta^2,
  e_t = e_(t-1)^2 (t = 2..n); e_n is the gadget's output.
* The product statement is a chain P_1 = d_0 d_1, P_j = P_(j-1) d_j, closing with
  P_(b-2) d_(b-1) = 0 (b = 1: d_0 * 1 = 0), with d_j written as the linear combination
  x_max - y_ij.
* GELU at fixed point: G = y^2 + 2^(F+1) y + 2^(2F+2) = 2^(2F+3) (x^2/8 + x/4 + 1/2) with
  x = y / 2^F, exact, one row y * y = G - 2^(F+1) y - 2^(2F+2).
* The gadget outputs are auxiliary (private) variables, like the intermediate
  activations of the paper's Transformer proofs; X, Y public or private as for the
  matmul circuits.

Variable layout of the gadget's auxiliary block (after the n - 1 prefix sums S_k):
  SoftMax, per row i of Y: x_max_i, then P_1 .. P_(b-2), then per entry j the 32 bits of
  d_ij, the 33 bits of u_ij, beta_ij, e_ij1 .. e_ijn (69 values per entry).
  GELU: G_ij row-major.
Rows after the n CRPC + PSQ rows: SoftMax, per row i: per entry j (32 bit rows, the d
recomposition row, 33 bit rows, the u recomposition row, the base row, n power rows),
then the row's product chain (max(1, b - 1) rows).  GELU: one row per entry, row-major.

Pins (tests/test_oracle_gadgets.py): the max of small vectors, a wrong x_max failing
either the product or the decomposition rows, exp outputs equal to (1 + x/8)^8 of the
rounded input as exact fractions and within 0.03 of e^x on [-8, 0], 0 below T, GELU
values equal to x^2/8 + x/4 + 1/2 exactly, tampered outputs failing, and Groth16
proofs over both circuits verifying.
"""
from .bn254 import R, fr_from_int

FRAC_BITS = 12          # F
EXP_SQUARINGS = 3       # n of (1 + x/2^n)^(2^n)
EXP_THRESHOLD = 1 << (FRAC_BITS + EXP_SQUARINGS)   # |T| at scale 2^F
D_BITS = 32             # bits of d = x_max - x_j
U_BITS = 33             # bits of u = |T| - d + 2^32
SOFTMAX_PER_ENTRY = D_BITS + U_BITS + 1 + EXP_SQUARINGS
SOFTMAX_ROWS_PER_ENTRY = D_BITS + 1 + U_BITS + 1 + 1 + EXP_SQUARINGS
GADGETS = ("softmax", "gelu")


# ---------------------------------------------------------------- counts and layout
def softmax_row_aux(b):
    """Auxiliary values of one row of b entries: x_max, P_1..P_(b-2), the entries."""
    return 1 + max(0, b - 2) + b * SOFTMAX_PER_ENTRY


def aux_count(gadget, a, b):
    return a * softmax_row_aux(b) if gadget == "softmax" else a * b


def row_count(gadget, a, b):
    return a * (b * SOFTMAX_ROWS_PER_ENTRY + max(1, b - 1)) if gadget == "softmax" else a * b


def _softmax_slots(base, b, i):
    """Variable indices of row i's block: (x_max, [P_1..P_(b-2)], per-entry base)."""
    start = base + i * softmax_row_aux(b)
    mx = start
    prods = list(range(start + 1, start + 1 + max(0, b - 2)))
    ent0 = start + 1 + max(0, b - 2)
    return mx, prods, [ent0 + j * SOFTMAX_PER_ENTRY for j in range(b)]


# ---------------------------------------------------------------- the approximations
def exp_approx_fixed(d):
    """(c, q, beta, [e_1..e_n]) for d = x_max - x >= 0 at scale 2^F (Sec. III-C exp)."""
    assert 0 <= d < (1 << D_BITS)
    c = 1 if d <= EXP_THRESHOLD else 0
    q = d >> EXP_SQUARINGS
    beta = c * ((1 << FRAC_BITS) - q)
    es, e = [], beta
    for _ in range(EXP_SQUARINGS):
        e = e * e
        es.append(e)
    return c, q, beta, es


def gelu_fixed(y):
    """G = 2^(2F+3) (x^2/8 + x/4 + 1/2) for x = y / 2^F (Sec. III-C GELU), an integer."""
    return y * y + (y << (FRAC_BITS + 1)) + (1 << (2 * FRAC_BITS + 2))


# ---------------------------------------------------------------- rows
def gadget_rows(gadget, a, b, yvar, aux0):
    """Constraint rows (A, B, C) of the gadget over Y (variable yvar(i, j)); the gadget's
    auxiliary block starts at variable aux0."""
    rows = []
    one = 0
    if gadget == "gelu":
        for i in range(a):
            for j in range(b):
                y = yvar(i, j)
                g = aux0 + i * b + j
                C = {g: 1, y: (R - (1 << (FRAC_BITS + 1))) % R, one: (R - (1 << (2 * FRAC_BITS + 2))) % R}
                rows.append(({y: 1}, {y: 1}, C))
        return rows
    for i in range(a):
        mx, prods, ents = _softmax_slots(aux0, b, i)
        for j in range(b):
            y = yvar(i, j)
            e0 = ents[j]
            dbits = list(range(e0, e0 + D_BITS))
            ubits = list(range(e0 + D_BITS, e0 + D_BITS + U_BITS))
            beta = e0 + D_BITS + U_BITS
            pows = list(range(beta + 1, beta + 1 + EXP_SQUARINGS))
            for v in dbits:                                  # bit rows of d
                rows.append(({v: 1}, {v: 1}, {v: 1}))
            A = {v: 1 << k for k, v in enumerate(dbits)}     # sum 2^k d_k - (x_max - y) = 0
            A[mx] = R - 1
            A[y] = 1
            rows.append((A, {one: 1}, {}))
            for v in ubits:                                  # bit rows of u
                rows.append(({v: 1}, {v: 1}, {v: 1}))
            A = {v: 1 << k for k, v in enumerate(ubits)}     # sum 2^k u_k - (|T| - d + 2^32) = 0
            A[one] = (R - EXP_THRESHOLD - (1 << D_BITS)) % R
            A[mx] = 1
            A[y] = R - 1
            rows.append((A, {one: 1}, {}))
            # beta = c (2^F - q), c = top bit of u, q = bits n.. of d
            Bq = {one: 1 << FRAC_BITS}
            for k in range(EXP_SQUARINGS, D_BITS):
                Bq[dbits[k]] = (R - (1 << (k - EXP_SQUARINGS))) % R
            rows.append(({ubits[-1]: 1}, Bq, {beta: 1}))
            prev = beta                                      # e_t = e_(t-1)^2
            for v in pows:
                rows.append(({prev: 1}, {prev: 1}, {v: 1}))
                prev = v
        # prod_j (x_max - y_ij) = 0 as a chain
        dlin = [{mx: 1, yvar(i, j): R - 1} for j in range(b)]
        if b == 1:
            rows.append((dlin[0], {one: 1}, {}))
        else:
            for j in range(1, b):
                A = dlin[0] if j == 1 else {prods[j - 2]: 1}
                C = {prods[j - 1]: 1} if j < b - 1 else {}
                rows.append((A, dlin[j], C))
    return rows


# ---------------------------------------------------------------- witness
def gadget_witness(gadget, Y, w, aux0, x_max=None):
    """Writes the gadget's auxiliary values for matmul output Y into w (from aux0).
    x_max: optional per-row override (to build a wrong witness for the pins)."""
    a, b = len(Y), len(Y[0])
    if gadget == "gelu":
        for i in range(a):
            for j in range(b):
                w[aux0 + i * b + j] = fr_from_int(gelu_fixed(Y[i][j]))
        return w
    for i in range(a):
        mx, prods, ents = _softmax_slots(aux0, b, i)
        m = max(Y[i]) if x_max is None else x_max[i]
        w[mx] = fr_from_int(m)
        P = None
        for j in range(b):
            d = m - Y[i][j]
            dm = d % (1 << D_BITS)           # a wrong x_max below the max leaves d < 0
            c, q, beta, es = exp_approx_fixed(dm)
            u = (EXP_THRESHOLD - dm + (1 << D_BITS)) % (1 << U_BITS)
            e0 = ents[j]
            for k in range(D_BITS):
                w[e0 + k] = (dm >> k) & 1
            for k in range(U_BITS):
                w[e0 + D_BITS + k] = (u >> k) & 1
            w[e0 + D_BITS + U_BITS] = beta % R
            for t, e in enumerate(es):
                w[e0 + D_BITS + U_BITS + 1 + t] = e % R
            df = fr_from_int(d)
            if j == 0:
                P = df
            else:
                P = P * df % R
                if 1 <= j <= b - 2:
                    w[prods[j - 1]] = P
    return w


def softmax_outputs(Y):
    """e_ij at scale 2^(F 2^n) for every entry (the gadget's outputs, plain integers)."""
    out = []
    for row in Y:
        m = max(row)
        out.append([exp_approx_fixed(m - y)[3][-1] for y in row])
    return out
