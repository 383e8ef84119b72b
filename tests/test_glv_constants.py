"""The GLV constants of the chain-mode scalar multiplications (csrc/glv.h), checked against
the mathematics with the oracle's curve arithmetic: lambda and beta are cube roots of unity
(mod r and mod p), phi(x, y) = (beta x, y) acts on G1 as multiplication by lambda, the two
basis vectors lie in the lattice {(x, y) : x + y lambda = 0 mod r} and span it (determinant
r), the rounding constants are floor(2^256 b / r), and the split k = k1 + k2 lambda (mod r)
written from the header's formulas gives halves below 2^127 on random and extreme k."""
import os
import random
import re

from oracle import bn254 as bn

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2504_12217_gb300", "csrc", "glv.h")


def _consts():
    text = open(HEADER).read()

    def limbs(name):
        m = re.search(r"constexpr uint64_t %s(?:\[\d\])? = \{?([^;}]*)\}?;" % name, text)
        vals = [int(v.strip().rstrip("ull"), 16) for v in m.group(1).split(",")]
        return sum(v << (64 * i) for i, v in enumerate(vals))

    beta_words = re.findall(r"i == \d \? (0x[0-9a-f]+)u", text)
    beta = sum(int(w, 16) << (32 * i) for i, w in enumerate(beta_words))
    lam = int(re.search(r"lambda = (0x[0-9a-f]+) \(mod r\)", text).group(1), 16)
    return lam, beta, {n: limbs(n) for n in ("GLV_A1", "GLV_B1", "GLV_A2", "GLV_B2", "GLV_G1", "GLV_G2")}


def test_cube_roots_and_endomorphism():
    lam, beta, _ = _consts()
    assert (lam * lam + lam + 1) % bn.R == 0 and lam not in (0, 1)
    assert (beta * beta + beta + 1) % bn.P == 0 and beta not in (0, 1)
    rng = random.Random(5)
    for P in (bn.G1_GEN, bn.g1_mul(bn.G1_GEN, rng.randrange(1, bn.R))):
        phi = (beta * P[0] % bn.P, P[1])
        assert bn.g1_on_curve(phi)
        assert phi == bn.g1_mul(P, lam)


def test_lattice_basis_and_rounding_constants():
    lam, _, c = _consts()
    a1, b1, a2, b2 = c["GLV_A1"], c["GLV_B1"], c["GLV_A2"], c["GLV_B2"]
    assert (a1 - b1 * lam) % bn.R == 0          # v1 = (a1, -b1)
    assert (a2 + b2 * lam) % bn.R == 0          # v2 = (a2, b2)
    assert a1 * b2 + a2 * b1 == bn.R            # det [[a1, -b1], [a2, b2]]
    assert c["GLV_G1"] == (b2 << 256) // bn.R
    assert c["GLV_G2"] == (b1 << 256) // bn.R


def test_split_reproduces_k_with_short_halves():
    lam, _, c = _consts()
    a1, b1, a2, b2, g1, g2 = (c[n] for n in ("GLV_A1", "GLV_B1", "GLV_A2", "GLV_B2", "GLV_G1", "GLV_G2"))
    rng = random.Random(6)
    ks = [0, 1, 2, bn.R - 1, bn.R - 2, bn.R // 2, 1 << 253, lam, bn.R - lam] + [rng.randrange(bn.R) for _ in range(5000)]
    for k in ks:
        c1, c2 = (k * g1) >> 256, (k * g2) >> 256
        k1 = k - c1 * a1 - c2 * a2
        k2 = c1 * b1 - c2 * b2
        assert (k1 + k2 * lam - k) % bn.R == 0
        assert abs(k1) < 1 << 127 and abs(k2) < 1 << 127
