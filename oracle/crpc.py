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

The ablation circuits of Sec. V (Table II) share the variable order one | X | Y | W |
auxiliary and differ in the auxiliary variables and rows (see CIRCUITS below); with
public_io = "none" only the constant one is public (l = 0), so X and Y join the private
variables and only one input-consistency row remains.

The gadget circuits of Sec. III-C ("crpc_psq_softmax", "crpc_psq_gelu") are the CRPC +
PSQ rows followed by the gadget's rows on Y (oracle/gadgets.py); their auxiliary block
follows the prefix sums.

Pins (tests/test_oracle_crpc.py, tests/test_oracle_circuits.py, tests/test_oracle_gadgets.py): the worked 3x2 . 2x2
example of Sec. III-A (golden exponents), the identity as integer polynomials in Z,
constraint satisfaction against a direct integer matmul, the constraint counts (n vs
a b n) and the PSQ left-wire counts (6 vs 3 for a 3-term dot product), the paper's two
negative examples, and for every circuit and public-input choice: satisfaction, a
tampered output failing, row and variable counts, and honest Groth16 proofs verifying.
"""
from . import gadgets
from .bn254 import R, fr_from_int

# Circuit variants of the paper's ablation (Sec. V, Table II):
#   "crpc_psq"  CRPC (Sec. III-A) with the PSQ chain (Sec. III-B)  -- the zkVC circuit
#   "crpc"      CRPC without PSQ: product variables p_k = a_k b_k and one summing row
#   "psq"       no CRPC, PSQ only: per output y_ij a prefix-sum chain over its n products
#   "vanilla"   no CRPC, no PSQ: one row per product x_ik w_kj = p_ijk (a b n rows, the
#               count Sec. III-A starts from) and one summing row per output
# and the public-input choice: "xy" (X and Y public, the default reading) or "none" (X and
# Y private too; only the constant one is public).
# The nonlinear gadgets of Sec. III-C on the matmul output (oracle/gadgets.py):
#   "crpc_psq_softmax"  the zkVC circuit, then per row of Y the max verification and the
#                       exponential approximation of SoftMax's numerators
#   "crpc_psq_gelu"     the zkVC circuit, then the GELU polynomial on every entry of Y
CIRCUITS = ("crpc_psq", "crpc", "psq", "vanilla", "crpc_psq_softmax", "crpc_psq_gelu")


def gadget_of(circuit):
    """The Sec. III-C gadget a circuit appends to the CRPC + PSQ rows, or None."""
    return {"crpc_psq_softmax": "softmax", "crpc_psq_gelu": "gelu"}.get(circuit)
PUBLIC_IO = ("xy", "none")


class Shape:
    def __init__(self, a, n, b, circuit="crpc_psq", public_io="xy"):
        assert a >= 1 and n >= 1 and b >= 1
        assert circuit in CIRCUITS and public_io in PUBLIC_IO
        self.a, self.n, self.b = a, n, b
        self.circuit, self.public_io = circuit, public_io
        self.n_io = a * n + a * b                          # entries of X and Y
        self.n_public = self.n_io if public_io == "xy" else 0   # l
        g = gadget_of(circuit)
        self.gadget = g
        if g:
            self.n_aux = n - 1 + gadgets.aux_count(g, a, b)
            self.n_circuit_rows = n + gadgets.row_count(g, a, b)
        else:
            self.n_aux = {"crpc_psq": n - 1, "crpc": n, "psq": a * b * (n - 1), "vanilla": a * b * n}[circuit]
            self.n_circuit_rows = {"crpc_psq": n, "crpc": n + 1, "psq": a * b * n,
                                   "vanilla": a * b * n + a * b}[circuit]
        self.n_vars = 1 + self.n_io + n * b + self.n_aux
        self.n_rows = self.n_circuit_rows + self.n_public + 1
        N = 1
        while N < self.n_rows:
            N *= 2
        self.domain = N

    # variable indices: one | X | Y | W | auxiliary
    def x(self, i, k):
        return 1 + i * self.n + k

    def y(self, i, j):
        return 1 + self.a * self.n + i * self.b + j

    def w(self, k, j):
        return 1 + self.n_io + k * self.b + j

    def aux(self, idx):
        return 1 + self.n_io + self.n * self.b + idx

    def s(self, k):
        """crpc_psq (and the gadget circuits): prefix sum S_k, k < n - 1."""
        return self.aux(k)

    def gadget_aux0(self):
        """First variable of the gadget's auxiliary block (after the n - 1 prefix sums)."""
        return self.aux(self.n - 1)

    def p(self, k):
        """crpc: product p_k = a_k b_k, k < n."""
        return self.aux(k)

    def s3(self, i, j, k):
        """psq: prefix sum S_ijk = sum_(k' <= k) x_ik' w_k'j, k < n - 1."""
        return self.aux((i * self.b + j) * (self.n - 1) + k)

    def p3(self, i, j, k):
        """vanilla: product p_ijk = x_ik w_kj."""
        return self.aux((i * self.b + j) * self.n + k)

    def __repr__(self):
        return f"Shape(a={self.a}, n={self.n}, b={self.b}, {self.circuit}, public {self.public_io})"


def build_r1cs(shape, z, with_input_rows=True):
    """Rows (A, B, C) as dicts {variable: Fr coefficient}, circuit rows first, then the
    input-consistency rows of the public variables (z is used by the CRPC circuits)."""
    a, n, b = shape.a, shape.n, shape.b
    rows = []
    if shape.circuit in ("crpc_psq", "crpc") or shape.gadget:
        for k in range(n):
            A = {shape.x(i, k): pow(z, i * b, R) for i in range(a)}
            B = {shape.w(k, j): pow(z, j, R) for j in range(b)}
            C = {}
            if shape.circuit == "crpc":
                C[shape.p(k)] = 1
            elif k < n - 1:
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
        if shape.circuit == "crpc":   # (p_0 + ... + p_(n-1)) * 1 = Y(z)
            C = {shape.y(i, j): pow(z, i * b + j, R) for i in range(a) for j in range(b)}
            rows.append(({shape.p(k): 1 for k in range(n)}, {0: 1}, C))
        if shape.gadget:              # Sec. III-C on Y
            rows += gadgets.gadget_rows(shape.gadget, a, b, shape.y, shape.gadget_aux0())
    else:
        for i in range(a):
            for j in range(b):
                for k in range(n):
                    A, B = {shape.x(i, k): 1}, {shape.w(k, j): 1}
                    if shape.circuit == "vanilla":
                        C = {shape.p3(i, j, k): 1}
                    else:
                        C = {shape.s3(i, j, k): 1} if k < n - 1 else {shape.y(i, j): 1}
                        if k >= 1:
                            C[shape.s3(i, j, k - 1)] = R - 1
                    rows.append((A, B, C))
        if shape.circuit == "vanilla":   # (p_ij0 + ... + p_ij(n-1)) * 1 = y_ij
            for i in range(a):
                for j in range(b):
                    rows.append(({shape.p3(i, j, k): 1 for k in range(n)}, {0: 1}, {shape.y(i, j): 1}))
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


def witness(shape, X, W, z, Y=None, x_max=None):
    """Full assignment w (length n_vars).  Y defaults to the true product X W.  x_max
    overrides the SoftMax gadget's per-row maxima (wrong witnesses for the pins)."""
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
    if shape.circuit in ("crpc_psq", "crpc") or shape.gadget:
        ak, bk = crpc_evaluations(X, W, z)
        if shape.circuit == "crpc":
            for k in range(n):
                w[shape.p(k)] = ak[k] * bk[k] % R
        else:
            S = 0
            for k in range(n - 1):                      # PSQ prefix sums (Sec. III-B)
                S = (S + ak[k] * bk[k]) % R
                w[shape.s(k)] = S
    else:
        for i in range(a):
            for j in range(b):
                acc = 0
                for k in range(n):
                    prod = X[i][k] * W[k][j]
                    if shape.circuit == "vanilla":
                        w[shape.p3(i, j, k)] = fr_from_int(prod)
                    elif k < n - 1:
                        acc += prod
                        w[shape.s3(i, j, k)] = fr_from_int(acc)
    if shape.gadget:                                    # Sec. III-C on Y
        gadgets.gadget_witness(shape.gadget, Y, w, shape.gadget_aux0(), x_max)
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
