"""The CRPC + PSQ rank-1 constraint system of a matrix product, built explicitly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages restated here:

* Sec. III-A (CRPC, general equation): for Y = X W with X of a x n, W of n x b,
      sum_{i,j} Z^(i b + j) y_ij = sum_k (sum_i Z^(i b) x_ik) (sum_j Z^j w_kj),
  so the product needs n multiplication constraints instead of a b n.
* Sec. III-B (PSQ): instead of product variables followed by one long addition, the
  constraint chain records prefix sums (a_7 = x00 w00, a_8 = a_7 + x01 w10, ...), so the
  final prefix sum is the result and each constraint has one product on its left wires.

Reading used for the combination (the paper defines PSQ on a scalar dot product only):
the prefix sums run over the n per-k CRPC products c_k = a_k b_k, with
a_k = sum_i z^(i b) x_ik and b_k = sum_j z^j w_kj, and the last constraint closes
against Y(z):

    row k < n-1 :  a_k * b_k = S_k - S_(k-1)       (S_(-1) = 0)
    row n-1     :  a_(n-1) * b_(n-1) = Y(z) - S_(n-2)     (n = 1: a_0 b_0 = Y(z))

z is one Fr element fixed at setup (the "random intermediate variable Z").

Variable order (libsnark style, one = variable 0, public inputs first):
    0                       the constant one
    1 .. a n                X, row-major           (public)
    then a b                Y, row-major           (public; l = a n + a b inputs)
    then n b                W, row-major           (private)
    then n - 1              S_0 .. S_(n-2)         (private)
After the n CRPC rows come l + 1 input-consistency rows n + i (i = 0..l) with A = [var i],
B = C = 0, the libsnark convention that binds the public inputs into the QAP.
The domain size is the next power of two >= n + l + 1.

Pins (tests/test_oracle_crpc.py): the worked 3x2 . 2x2 example of Sec. III-A (golden
exponents), the identity as integer polynomials in Z, constraint satisfaction against a
direct integer matmul, the constraint counts (n vs a b n) and the PSQ left-wire counts
(6 vs 3 for a 3-term dot product), and the paper's two negative examples.
"""
from .bn254 import R, fr_from_int


class Shape:
    def __init__(self, a, n, b):
        assert a >= 1 and n >= 1 and b >= 1
        self.a, self.n, self.b = a, n, b
        self.n_public = a * n + a * b                    # l
        self.n_vars = 1 + self.n_public + n * b + (n - 1)
        self.n_rows = n + self.n_public + 1
        N = 1
        while N < self.n_rows:
            N *= 2
        self.domain = N

    # variable indices
    def x(self, i, k):
        return 1 + i * self.n + k

    def y(self, i, j):
        return 1 + self.a * self.n + i * self.b + j

    def w(self, k, j):
        return 1 + self.n_public + k * self.b + j

    def s(self, k):
        return 1 + self.n_public + self.n * self.b + k

    def __repr__(self):
        return f"Shape(a={self.a}, n={self.n}, b={self.b})"


def build_r1cs(shape, z, with_input_rows=True):
    """Rows (A, B, C) as dicts {variable: Fr coefficient}, CRPC rows first."""
    a, n, b = shape.a, shape.n, shape.b
    rows = []
    for k in range(n):
        A = {shape.x(i, k): pow(z, i * b, R) for i in range(a)}
        B = {shape.w(k, j): pow(z, j, R) for j in range(b)}
        C = {}
        if k < n - 1:
            C[shape.s(k)] = 1
            if k >= 1:
                C[shape.s(k - 1)] = R - 1
        else:
            for i in range(a):
                for j in range(b):
                    C[shape.y(i, j)] = pow(z, i * b + j, R)
            if n >= 2:
                C[shape.s(n - 2)] = R - 1
        rows.append((A, B, C))
    if with_input_rows:
        for i in range(shape.n_public + 1):
            rows.append(({i: 1}, {}, {}))
    return rows


def matmul_int(X, W):
    a, n, b = len(X), len(W), len(W[0])
    return [[sum(X[i][k] * W[k][j] for k in range(n)) for j in range(b)] for i in range(a)]


def crpc_evaluations(X, W, z):
    """a_k = sum_i z^(ib) x_ik and b_k = sum_j z^j w_kj over Fr (Sec. III-A)."""
    a, n, b = len(X), len(W), len(W[0])
    ak = [sum(pow(z, i * b, R) * fr_from_int(X[i][k]) for i in range(a)) % R for k in range(n)]
    bk = [sum(pow(z, j, R) * fr_from_int(W[k][j]) for j in range(b)) % R for k in range(n)]
    return ak, bk


def crpc_y_at_z(Y, z):
    a, b = len(Y), len(Y[0])
    return sum(pow(z, i * b + j, R) * fr_from_int(Y[i][j]) for i in range(a) for j in range(b)) % R


def witness(shape, X, W, z, Y=None):
    """Full assignment w (length n_vars).  Y defaults to the true product X W."""
    a, n, b = shape.a, shape.n, shape.b
    if Y is None:
        Y = matmul_int(X, W)
    w = [0] * shape.n_vars
    w[0] = 1
    for i in range(a):
        for k in range(n):
            w[shape.x(i, k)] = fr_from_int(X[i][k])
    for i in range(a):
        for j in range(b):
            w[shape.y(i, j)] = fr_from_int(Y[i][j])
    for k in range(n):
        for j in range(b):
            w[shape.w(k, j)] = fr_from_int(W[k][j])
    ak, bk = crpc_evaluations(X, W, z)
    S = 0
    for k in range(n - 1):                      # PSQ prefix sums (Sec. III-B)
        S = (S + ak[k] * bk[k]) % R
        w[shape.s(k)] = S
    return w


def dot(row, w):
    return sum(c * w[v] for v, c in row.items()) % R


def unsatisfied_rows(rows, w):
    """Indices k with <A_k, w> <B_k, w> != <C_k, w>."""
    bad = []
    for k, (A, B, C) in enumerate(rows):
        if dot(A, w) * dot(B, w) % R != dot(C, w):
            bad.append(k)
    return bad


# ---------------------------------------------------------------- counting pins
def left_wire_count(rows):
    """Number of (row, variable) entries of the A matrix: the "left wires" of Sec. III-B."""
    return sum(len(A) for A, _, _ in rows)


def dot_product_rows_without_psq(n):
    """Sec. III-B, Fig. 5(a): one constraint per product p_k = x_k w_k, then one constraint
    (p_0 + ... + p_(n-1)) * 1 = y.  Variables: 0 one, x_k = 1+k, w_k = 1+n+k,
    p_k = 1+2n+k, y = 1+3n."""
    rows = []
    for k in range(n):
        rows.append(({1 + k: 1}, {1 + n + k: 1}, {1 + 2 * n + k: 1}))
    rows.append(({1 + 2 * n + k: 1 for k in range(n)}, {0: 1}, {1 + 3 * n: 1}))
    return rows


def vanilla_matmul_constraint_count(a, n, b):
    """Sec. III-A: one constraint per individual multiplication x_ik w_kj."""
    return a * b * n
