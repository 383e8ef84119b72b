"""The G2 endomorphism constants of the variable-base G2 MSM (csrc/glv.h), checked against
the mathematics with the oracle's curve arithmetic: gx and gy are xi^((p-1)/3) and
xi^((p-1)/2) in Fp2 (recomputed here by the oracle's Fp2 power), psi(x, y) = (conj(x) gx,
conj(y) gy) maps G2 to itself and acts on it as multiplication by lambda2 = 6 u^2 = p mod r,
g = floor(2^256 / lambda2), and the split written from the header's formula (quotient
estimate, one correction) gives k = k1 + k2 lambda2 with 0 <= k1, k2 < 2^127 on random
and extreme k."""
import os
import random
import re

from oracle import bn254 as bn

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2504_12217_gb300", "csrc", "glv.h")


def _consts():
    text = open(HEADER).read()

    def u64(name):
        m = re.search(r"constexpr uint64_t %s\[\d\] = \{([^}]*)\};" % name, text)
        vals = [int(v.strip().rstrip("ull"), 16) for v in m.group(1).split(",")]
        return sum(v << (64 * i) for i, v in enumerate(vals))

    def fp2(fn):
        body = re.search(r"uint32_t %s\(int c, int i\) \{(.*?)return" % fn, text, re.S).group(1)
        words = [int(w, 16) for w in re.findall(r"0x([0-9a-f]+)u", body)]
        assert len(words) == 16
        return (sum(w << (32 * i) for i, w in enumerate(words[:8])),
                sum(w << (32 * i) for i, w in enumerate(words[8:])))

    return u64("PSI_LAMBDA"), u64("PSI_G"), fp2("psi_gx_limb"), fp2("psi_gy_limb")


def _psi(Q, gx, gy):
    (x0, x1), (y0, y1) = Q
    return (bn.f2_mul((x0, (-x1) % bn.P), gx), bn.f2_mul((y0, (-y1) % bn.P), gy))


def test_constants_are_the_frobenius_twist_coefficients():
    lam, g, gx, gy = _consts()
    assert gx == bn.f2_pow(bn.XI, (bn.P - 1) // 3)
    assert gy == bn.f2_pow(bn.XI, (bn.P - 1) // 2)
    assert lam == 6 * bn.U * bn.U == bn.P % bn.R
    assert g == (1 << 256) // lam


def test_psi_is_multiplication_by_lambda2_on_g2():
    lam, _, gx, gy = _consts()
    rng = random.Random(11)
    for Q in (bn.G2_GEN, bn.g2_mul(bn.G2_GEN, rng.randrange(1, bn.R))):
        pq = _psi(Q, gx, gy)
        assert bn.g2_on_curve(pq)
        assert pq == bn.g2_mul(Q, lam)


def test_split_reproduces_k_with_short_nonnegative_halves():
    lam, g, _, _ = _consts()
    rng = random.Random(12)
    ks = [0, 1, lam - 1, lam, lam + 1, 2 * lam, bn.R - 1, bn.R - 2, bn.R // 2] + [rng.randrange(bn.R) for _ in range(5000)]
    for k in ks:
        q = (k * g) >> 256
        k1 = k - q * lam
        assert 0 <= k1 < 2 * lam
        if k1 >= lam:
            k1, q = k1 - lam, q + 1
        assert k1 + q * lam == k
        assert 0 <= k1 < 1 << 127 and 0 <= q < 1 << 127
