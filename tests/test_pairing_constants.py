"""Identities the GPU pairing code relies on (no GPU needed): the BN decomposition of the
hard part of the final exponent into powers of p with coefficients polynomial in u, the
bit length of the optimal ate loop scalar 6u + 2, and 6 | p - 1 (the Frobenius constants
xi^(m (p^k - 1)/6))."""
from oracle import bn254 as bn


def test_final_exponent_decomposition():
    """(p^4 - p^2 + 1)/r = p^3 + l2 p^2 + l1 p + l0 with l2 = 6u^2 + 1,
    l1 = -36u^3 - 18u^2 - 12u + 1, l0 = -36u^3 - 30u^2 - 18u - 2 (BN curves), and the
    Miller-loop scalar 6u + 2 has 65 bits."""
    u, p, r = bn.U, bn.P, bn.R
    hard, rem = divmod(p ** 4 - p ** 2 + 1, r)
    assert rem == 0
    assert hard == p ** 3 + (6 * u * u + 1) * p ** 2 + (-36 * u ** 3 - 18 * u * u - 12 * u + 1) * p + \
        (-36 * u ** 3 - 30 * u * u - 18 * u - 2)
    assert (6 * u + 2).bit_length() == 65 and (p - 1) % 6 == 0
