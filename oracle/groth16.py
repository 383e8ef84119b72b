"""Groth16 over the CRPC + PSQ QAP: setup, prove, verify, and a closed-form proof.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

zkVC Sec. II describes a ZKP construction as Gen / Prove / Verify, and Sec. IV runs the
groth16 backend of libsnark.  This module restates the libsnark-style presentation of
Groth16 on the R1CS of ``oracle.crpc``:

QAP (Sec. II: R1CS encoded by polynomial interpolation).  For each variable i,
A_i(x) = sum_k A_(k,i) L_k(x) with L_k the Lagrange basis of H = {omega^k}, k < N;
t(x) = x^N - 1.

Setup, with toxic waste (tau, alpha, beta, gamma, delta):
    pk: [alpha]1, [beta]1, [beta]2, [delta]1, [delta]2,
        A-query  [A_i(tau)]1             for the variables in the support of A
        B-query  [B_i(tau)]1, [B_i(tau)]2 for the variables in the support of B
        L-query  [(beta A_i + alpha B_i + C_i)(tau) / delta]1   for private i
        H-query  [tau^j t(tau) / delta]1                        for j = 0 .. N-2
    vk: e([alpha]1, [beta]2), [gamma]2, [delta]2,
        IC_i = [(beta A_i + alpha B_i + C_i)(tau) / gamma]1      for i = 0 .. l

Prove, with the assignment w and prover randomness (r, s):
    A = [alpha]1 + sum_i w_i [A_i]1 + r [delta]1
    B = [beta]2 + sum_i w_i [B_i]2 + s [delta]2    (B1 the same in G1)
    C = sum_priv w_i L_i + sum_j h_j H_j + s A + r B1 - r s [delta]1
where h = (A(x) B(x) - C(x)) / t(x) is computed through the domain evaluations, INTT,
coset NTT, pointwise division by t(g omega^k) = g^N - 1, and coset INTT (``oracle.ntt``).

Verify: e(A, B) = e(alpha, beta) e(IC_0 + sum_i x_i IC_i, gamma) e(C, delta).

Pins (tests/test_oracle_groth16.py): L_k(tau) against the product formula and the
interpolation identity; h t = A B - C at a random point and h[N-1] = 0; honest proofs
verify; a flipped y_ij, a perturbed proof element and swapped A/C do not; the naive
proof equals the closed-form proof computed from the toxic waste.
"""
from . import bn254 as bn
from .bn254 import R
from . import ntt as nt
from . import crpc
from .pairing import pairing, pairing_product_is_one


# ---------------------------------------------------------------- QAP
def lagrange_at(tau, N, rows=None):
    """L_k(tau) = (tau^N - 1) omega^k / (N (tau - omega^k)) for k < rows (default N).

    Closed form of prod_(j != k) (tau - omega^j)/(omega^k - omega^j), using that the
    derivative of x^N - 1 at omega^k is N omega^(-k).
    """
    rows = N if rows is None else rows
    omega = bn.fr_root_of_unity(N)
    tN = (pow(tau, N, R) - 1) % R
    coef = tN * pow(N, -1, R) % R
    out = []
    wk = 1
    for _ in range(rows):
        out.append(coef * wk % R * pow((tau - wk) % R, -1, R) % R)
        wk = wk * omega % R
    return out


def lagrange_at_product(tau, N, k):
    """Textbook product formula for one L_k(tau) (used by the pin of ``lagrange_at``)."""
    omega = bn.fr_root_of_unity(N)
    wk = pow(omega, k, R)
    num, den = 1, 1
    for j in range(N):
        if j == k:
            continue
        wj = pow(omega, j, R)
        num = num * (tau - wj) % R
        den = den * (wk - wj) % R
    return num * pow(den, -1, R) % R


def qap_at(rows, n_vars, Lk):
    """Per-variable A_i(tau), B_i(tau), C_i(tau) and their structural supports."""
    At, Bt, Ct = [0] * n_vars, [0] * n_vars, [0] * n_vars
    sA, sB, sC = set(), set(), set()
    for k, (A, B, C) in enumerate(rows):
        L = Lk[k]
        for v, c in A.items():
            At[v] = (At[v] + c * L) % R
            sA.add(v)
        for v, c in B.items():
            Bt[v] = (Bt[v] + c * L) % R
            sB.add(v)
        for v, c in C.items():
            Ct[v] = (Ct[v] + c * L) % R
            sC.add(v)
    return At, Bt, Ct, sorted(sA), sorted(sB), sorted(sC)


# ---------------------------------------------------------------- keys
class ProvingKey:
    pass


class VerifyingKey:
    pass


def setup(shape, toxic):
    """Groth16 Gen for the CRPC + PSQ circuit of ``shape``.

    toxic = (tau, alpha, beta, gamma, delta, z); z is the CRPC point of Sec. III-A.
    """
    tau, alpha, beta, gamma, delta, z = [t % R for t in toxic]
    N = shape.domain
    assert pow(tau, N, R) != 1 and 0 not in (alpha, beta, gamma, delta)
    rows = crpc.build_r1cs(shape, z)
    Lk = lagrange_at(tau, N, len(rows))
    At, Bt, Ct, sA, sB, _ = qap_at(rows, shape.n_vars, Lk)
    G1, G2 = bn.G1_GEN, bn.G2_GEN
    l = shape.n_public
    di, gi = pow(delta, -1, R), pow(gamma, -1, R)
    tt = (pow(tau, N, R) - 1) % R

    pk = ProvingKey()
    pk.shape, pk.z, pk.rows = shape, z, rows
    pk.alpha1, pk.beta1, pk.beta2 = bn.g1_mul(G1, alpha), bn.g1_mul(G1, beta), bn.g2_mul(G2, beta)
    pk.delta1, pk.delta2 = bn.g1_mul(G1, delta), bn.g2_mul(G2, delta)
    pk.A_vars = sA
    pk.A = [bn.g1_mul(G1, At[i]) for i in sA]
    pk.B_vars = sB
    pk.B1 = [bn.g1_mul(G1, Bt[i]) for i in sB]
    pk.B2 = [bn.g2_mul(G2, Bt[i]) for i in sB]
    pk.L_vars = list(range(l + 1, shape.n_vars))
    pk.L = [bn.g1_mul(G1, (beta * At[i] + alpha * Bt[i] + Ct[i]) * di) for i in pk.L_vars]
    pk.H = [bn.g1_mul(G1, pow(tau, j, R) * tt % R * di) for j in range(N - 1)]

    vk = VerifyingKey()
    vk.shape = shape
    vk.alpha_beta = pairing(pk.alpha1, pk.beta2)
    vk.alpha1, vk.beta2 = pk.alpha1, pk.beta2
    vk.gamma2, vk.delta2 = bn.g2_mul(G2, gamma), pk.delta2
    vk.IC = [bn.g1_mul(G1, (beta * At[i] + alpha * Bt[i] + Ct[i]) * gi) for i in range(l + 1)]
    return pk, vk


# ---------------------------------------------------------------- quotient
def domain_evaluations(rows, w, N):
    """<A_k, w>, <B_k, w>, <C_k, w> for each row k, zero-padded to N."""
    Aev, Bev, Cev = [0] * N, [0] * N, [0] * N
    for k, (A, B, C) in enumerate(rows):
        Aev[k], Bev[k], Cev[k] = crpc.dot(A, w), crpc.dot(B, w), crpc.dot(C, w)
    return Aev, Bev, Cev


def quotient(Aev, Bev, Cev):
    """h with h t = A B - C, through the coset gH (g = 5): N - 1 coefficients h_0..h_(N-2).

    Returns the full length-N coefficient list; h[N-1] = 0 is asserted by the caller.
    """
    N = len(Aev)
    a, b, c = nt.intt(Aev), nt.intt(Bev), nt.intt(Cev)
    ae, be, ce = nt.coset_ntt(a), nt.coset_ntt(b), nt.coset_ntt(c)
    zinv = pow((pow(bn.FR_GEN, N, R) - 1) % R, -1, R)   # 1 / t(g omega^k)
    hev = [((x * y - z) * zinv) % R for x, y, z in zip(ae, be, ce)]
    return nt.coset_intt(hev), (a, b, c)


# ---------------------------------------------------------------- prove / verify
def prove(pk, X, W, r, s, Y=None):
    """Groth16 Prove (naive MSMs).  Returns (proof dict, Y, h)."""
    shape = pk.shape
    N = shape.domain
    if Y is None:
        Y = crpc.matmul_int(X, W)
    w = crpc.witness(shape, X, W, pk.z, Y)
    Aev, Bev, Cev = domain_evaluations(pk.rows, w, N)
    h, _ = quotient(Aev, Bev, Cev)
    assert h[N - 1] == 0, "quotient has degree N-1: the witness does not satisfy the QAP"
    r %= R
    s %= R
    A = bn.g1_add(bn.g1_add(pk.alpha1, bn.g1_msm(pk.A, [w[i] for i in pk.A_vars])),
                  bn.g1_mul(pk.delta1, r))
    B2 = bn.g2_add(bn.g2_add(pk.beta2, bn.g2_msm(pk.B2, [w[i] for i in pk.B_vars])),
                   bn.g2_mul(pk.delta2, s))
    B1 = bn.g1_add(bn.g1_add(pk.beta1, bn.g1_msm(pk.B1, [w[i] for i in pk.B_vars])),
                   bn.g1_mul(pk.delta1, s))
    C = bn.g1_msm(pk.L, [w[i] for i in pk.L_vars])
    C = bn.g1_add(C, bn.g1_msm(pk.H, h[:N - 1]))
    C = bn.g1_add(C, bn.g1_mul(A, s))
    C = bn.g1_add(C, bn.g1_mul(B1, r))
    C = bn.g1_add(C, bn.g1_neg(bn.g1_mul(pk.delta1, r * s)))
    return {"A": A, "B": B2, "C": C}, Y, h


def proof_bytes(proof):
    """A (64) || B (128) || C (64) = 256 bytes, canonical little-endian affine."""
    return bn.g1_bytes(proof["A"]) + bn.g2_bytes(proof["B"]) + bn.g1_bytes(proof["C"])


def proof_from_bytes(bs):
    return {"A": bn.g1_from_bytes(bs[:64]), "B": bn.g2_from_bytes(bs[64:192]),
            "C": bn.g1_from_bytes(bs[192:256])}


def public_inputs(shape, X, Y):
    """x_1..x_l = X row-major then Y row-major, mapped to Fr (none when X and Y are
    private)."""
    if shape.n_public == 0:
        return []
    xs = [bn.fr_from_int(X[i][k]) for i in range(shape.a) for k in range(shape.n)]
    xs += [bn.fr_from_int(Y[i][j]) for i in range(shape.a) for j in range(shape.b)]
    return xs


def verify(vk, X, Y, proof):
    """Groth16 Verify: e(A,B) = e(alpha,beta) e(IC(x),gamma) e(C,delta)."""
    xs = public_inputs(vk.shape, X, Y)
    ic = vk.IC[0]
    ic = bn.g1_add(ic, bn.g1_msm(vk.IC[1:], xs))
    A, B, C = proof["A"], proof["B"], proof["C"]
    for Pt in (A, C):
        if not bn.g1_on_curve(Pt):
            return False
    if not bn.g2_on_curve(B):
        return False
    # e(A,B) e(-alpha,beta) e(-IC,gamma) e(-C,delta) = 1 is the same equation with one
    # shared final exponentiation.
    return pairing_product_is_one([(A, B), (bn.g1_neg(vk.alpha1), vk.beta2),
                                   (bn.g1_neg(ic), vk.gamma2), (bn.g1_neg(C), vk.delta2)])


# ---------------------------------------------------------------- closed form
def closed_form_proof(shape, toxic, X, W, r, s, Y=None):
    """The proof computed from the toxic waste in the exponent.

    Every pk point is [scalar]G, so each MSM equals [sum of scalar products]G and
        A = [alpha + sum w_i A_i(tau) + r delta]1
        B = [beta  + sum w_i B_i(tau) + s delta]2
        C = [(sum_priv w_i (beta A_i + alpha B_i + C_i)(tau) + h(tau) t(tau)) / delta
             + s a + r b - r s delta]1,     with h(tau) t(tau) = A(tau) B(tau) - C(tau).
    Equal to ``prove`` when the witness satisfies the R1CS (pinned on small shapes); needs
    O(rows + vars) field operations and three scalar multiplications, so it checks
    full-size proofs.
    """
    tau, alpha, beta, gamma, delta, z = [t % R for t in toxic]
    r %= R
    s %= R
    N = shape.domain
    if Y is None:
        Y = crpc.matmul_int(X, W)
    rows = crpc.build_r1cs(shape, z)
    w = crpc.witness(shape, X, W, z, Y)
    Lk = lagrange_at(tau, N, len(rows))
    At, Bt, Ct, _, _, _ = qap_at(rows, shape.n_vars, Lk)
    Aw = sum(wi * ai for wi, ai in zip(w, At)) % R
    Bw = sum(wi * bi for wi, bi in zip(w, Bt)) % R
    Cw = sum(wi * ci for wi, ci in zip(w, Ct)) % R
    a_s = (alpha + Aw + r * delta) % R
    b_s = (beta + Bw + s * delta) % R
    l = shape.n_public
    priv = sum(w[i] * (beta * At[i] + alpha * Bt[i] + Ct[i]) for i in range(l + 1, shape.n_vars))
    c_s = ((priv + Aw * Bw - Cw) * pow(delta, -1, R) + s * a_s + r * b_s - r * s * delta) % R
    return {"A": bn.g1_mul(bn.G1_GEN, a_s), "B": bn.g2_mul(bn.G2_GEN, b_s),
            "C": bn.g1_mul(bn.G1_GEN, c_s)}, Y


def pk_entry_scalars(shape, toxic, query, indices):
    """Scalars s with pk[query][idx] = [s]G for the given entry indices.

    query in {"A", "B", "L", "H"}; indices are positions in the oracle's pk lists.
    Used to check individual pk entries of a full-size key without a full setup.
    """
    tau, alpha, beta, gamma, delta, z = [t % R for t in toxic]
    N = shape.domain
    if query == "H":
        tt = (pow(tau, N, R) - 1) * pow(delta, -1, R) % R
        return [pow(tau, j, R) * tt % R for j in indices]
    rows = crpc.build_r1cs(shape, z)
    Lk = lagrange_at(tau, N, len(rows))
    At, Bt, Ct, sA, sB, _ = qap_at(rows, shape.n_vars, Lk)
    l = shape.n_public
    if query == "A":
        return [At[sA[i]] for i in indices]
    if query == "B":
        return [Bt[sB[i]] for i in indices]
    if query == "L":
        di = pow(delta, -1, R)
        return [(beta * At[l + 1 + i] + alpha * Bt[l + 1 + i] + Ct[l + 1 + i]) * di % R
                for i in indices]
    if query == "IC":
        gi = pow(gamma, -1, R)
        return [(beta * At[i] + alpha * Bt[i] + Ct[i]) * gi % R for i in indices]
    raise ValueError(query)
