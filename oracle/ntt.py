"""Number-theoretic transforms over Fr, textbook forms.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The QAP quotient h(x) (zkVC Sec. II: R1CS encoded as a QAP by interpolation over a
domain; Sec. III-A notes that the quotient polynomial dominates the CRPC savings) is
computed through evaluations on the domain H = <omega_N> and on the coset gH:

* ``ntt(a)[k]    = sum_i a_i omega^(i k)``               (natural order in and out)
* ``intt(v)[i]   = N^-1 sum_k v_k omega^(-i k)``
* ``coset_ntt(a) = ntt(a_i g^i)``                        (evaluations at g omega^k)
* ``coset_intt(v)_i = intt(v)_i g^-i``

``ntt`` is the recursive radix-2 Cooley-Tukey split into even and odd coefficients.
``dft`` is the O(N^2) definition and pins it (tests/test_oracle_ntt.py), together with
the round trip and the convolution theorem against schoolbook polynomial products.
"""
from .bn254 import R, FR_GEN, fr_root_of_unity


def dft(a, omega):
    """O(N^2) evaluation of the polynomial with coefficients a at omega^k, k < N."""
    n = len(a)
    out = []
    for k in range(n):
        wk = pow(omega, k, R)
        acc = 0
        x = 1
        for i in range(n):
            acc += a[i] * x
            x = x * wk % R
        out.append(acc % R)
    return out


def _ct(a, omega):
    n = len(a)
    if n == 1:
        return [a[0] % R]
    w2 = omega * omega % R
    even = _ct(a[0::2], w2)
    odd = _ct(a[1::2], w2)
    half = n // 2
    out = [0] * n
    w = 1
    for k in range(half):
        t = w * odd[k] % R
        out[k] = (even[k] + t) % R
        out[k + half] = (even[k] - t) % R
        w = w * omega % R
    return out


def ntt(a):
    n = len(a)
    return _ct(list(a), fr_root_of_unity(n))


def intt(v):
    n = len(v)
    w_inv = pow(fr_root_of_unity(n), -1, R)
    n_inv = pow(n, -1, R)
    return [x * n_inv % R for x in _ct(list(v), w_inv)]


def coset_ntt(a, g=FR_GEN):
    shifted = []
    gi = 1
    for x in a:
        shifted.append(x * gi % R)
        gi = gi * g % R
    return ntt(shifted)


def coset_intt(v, g=FR_GEN):
    coeffs = intt(v)
    g_inv = pow(g, -1, R)
    out = []
    gi = 1
    for x in coeffs:
        out.append(x * gi % R)
        gi = gi * g_inv % R
    return out


def poly_eval(coeffs, x):
    """Horner evaluation of sum_i c_i x^i mod r."""
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * x + c) % R
    return acc


def poly_mul_schoolbook(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] = (out[i + j] + x * y) % R
    return out
