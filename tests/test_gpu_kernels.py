"""GPU parity of the kernel layer against the oracle: Montgomery products, NTTs, MSMs.

Bit-exact comparisons (field and group results are exact)."""
import random

import numpy as np
import pytest

from oracle import bn254 as bn
from oracle import ntt as ont
from tests import _util

pytestmark = pytest.mark.gpu

P, R = bn.P, bn.R


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _edge(m):
    return [0, 1, 2, m - 1, m - 2, (m - 1) // 2, (m + 1) // 2, 1 << 128, (1 << 253) % m, 0xFFFFFFFF,
            1 << 32, (1 << 64) - 1]


@pytest.mark.parametrize("name,mod", [("fr", R), ("fp", P)])
def test_prime_field_mul(nv, name, mod):
    rng = random.Random(11)
    a = _edge(mod) + [rng.randrange(mod) for _ in range(4000)]
    b = list(reversed(_edge(mod))) + [rng.randrange(mod) for _ in range(4000)]
    fn = getattr(nv, f"zkvc_{name}_mul")
    out = fn(_util.to_cuda(_util.ints_to_u8(a)), _util.to_cuda(_util.ints_to_u8(b)))
    got = _util.u8_to_ints(out.cpu().numpy())
    assert got == [x * y % mod for x, y in zip(a, b)]


@pytest.mark.parametrize("name,mod", [("fr", R), ("fp", P)])
def test_prime_field_inv(nv, name, mod):
    """a^-1 against its definition (a a^-1 = 1; 0 -> 0).  The device inverts the integer
    y = a 2^256 mod m (the Montgomery form of a), so the inputs include a = y 2^-256 for
    the y that stress the binary GCD: tiny and all-ones values, powers of two, m - 1, and
    ratios of consecutive Fibonacci numbers (the most subtraction steps)."""
    rng = random.Random(12)
    rinv = pow(1 << 256, -1, mod)
    fib = [1, 2]
    while fib[-1] < mod:
        fib.append(fib[-1] + fib[-2])
    ys = [1, 2, 3, mod - 1, mod - 2, (mod - 1) // 2, (mod + 1) // 2, (1 << 253) - 1, 1 << 253, (1 << 64) - 1,
          1 << 64, (1 << 31) - 1, 1 << 31] + [f for f in fib[-8:] if f < mod] + [1 << k for k in range(0, 254, 7)]
    ys += [rng.randrange(1, 1 << rng.randrange(1, 254)) for _ in range(1000)]
    a = [0] + _edge(mod) + [y * rinv % mod for y in ys] + [rng.randrange(mod) for _ in range(3000)]
    out = getattr(nv, f"zkvc_{name}_inv")(_util.to_cuda(_util.ints_to_u8(a)))
    got = _util.u8_to_ints(out.cpu().numpy())
    for x, g in zip(a, got):
        assert g == (pow(x, -1, mod) if x else 0), x


def test_fp2_mul(nv):
    rng = random.Random(12)
    n = 2000
    a = [(rng.randrange(P), rng.randrange(P)) for _ in range(n)] + [(0, 0), (1, 0), (0, 1), (P - 1, P - 1)]
    b = [(rng.randrange(P), rng.randrange(P)) for _ in range(n)] + [(5, 7), (0, 1), (0, 1), (P - 1, 1)]
    enc = lambda xs: _util.ints_to_u8([c for z in xs for c in z]).reshape(len(xs), 64)
    out = nv.zkvc_fp2_mul(_util.to_cuda(enc(a)), _util.to_cuda(enc(b)))
    flat = _util.u8_to_ints(out.cpu().numpy().reshape(-1, 32))
    got = [(flat[2 * i], flat[2 * i + 1]) for i in range(len(a))]
    assert got == [bn.f2_mul(x, y) for x, y in zip(a, b)]


KINDS = {
    0: ont.ntt,
    1: ont.intt,
    2: ont.coset_ntt,
    3: ont.coset_intt,
}


@pytest.mark.parametrize("log_n", [1, 2, 3, 5, 8, 10, 11, 12, 13])
def test_ntt_all_kinds(nv, log_n):
    rng = random.Random(100 + log_n)
    n = 1 << log_n
    a = [rng.randrange(R) for _ in range(n)]
    if log_n == 5:
        a[:4] = [0, R - 1, 1, 0]
    for kind, ref in KINDS.items():
        t = _util.to_cuda(_util.ints_to_u8(a))
        nv.zkvc_ntt(t, kind)
        assert _util.u8_to_ints(t.cpu().numpy()) == ref(a), f"kind {kind}"


def test_ntt_2_16_parity(nv):
    rng = random.Random(216)
    n = 1 << 16
    a = [rng.randrange(R) for _ in range(n)]
    t = _util.to_cuda(_util.ints_to_u8(a))
    nv.zkvc_ntt(t, 0)
    assert _util.u8_to_ints(t.cpu().numpy()) == ont.ntt(a)
    nv.zkvc_ntt(t, 1)
    assert _util.u8_to_ints(t.cpu().numpy()) == a


@pytest.mark.parametrize("log_n", [17, 20, 22])
def test_ntt_large_sampled(nv, log_n):
    """Round trips at any size, plus sampled outputs computed one by one."""
    import torch
    n = 1 << log_n
    g = torch.Generator().manual_seed(log_n)
    raw = torch.randint(0, 256, (n, 32), dtype=torch.uint8, generator=g)
    raw[:, 31] &= 0x0F                      # < 2^252 < r: canonical
    x = raw.cuda()
    t = x.clone()
    nv.zkvc_ntt(t, 2)
    nv.zkvc_ntt(t, 3)
    assert torch.equal(t, x)
    t = x.clone()
    nv.zkvc_ntt(t, 0)
    out = t.cpu().numpy()
    a = _util.u8_to_ints(raw.numpy())
    w = bn.fr_root_of_unity(n)
    for k in (0, 1, n // 2 + 3, n - 1):
        wk = pow(w, k, R)
        acc, xp = 0, 1
        for ai in a:
            acc += ai * xp
            xp = xp * wk % R
        assert _util.u8_to_ints(out[k:k + 1])[0] == acc % R
    nv.zkvc_ntt(t, 1)
    assert torch.equal(t, x)


def _rand_g1(rng, n):
    return [bn.g1_mul(bn.G1_GEN, rng.randrange(1, R)) for _ in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 17, 256, 1500])
def test_msm_g1_random(nv, n):
    rng = random.Random(n)
    pts = _rand_g1(rng, n)
    sc = [rng.randrange(R) for _ in range(n)]
    got = nv.zkvc_msm_g1(_util.to_cuda(_util.g1_rows(pts)), _util.to_cuda(_util.ints_to_u8(sc)))
    assert got == bn.g1_bytes(bn.g1_msm(pts, sc))


def test_msm_g1_edge_cases(nv):
    rng = random.Random(5)
    P0 = bn.g1_mul(bn.G1_GEN, 12345)
    P1 = bn.g1_mul(bn.G1_GEN, 999)
    cases = [
        ([P0, P1], [0, 0]),                                # all-zero scalars -> infinity
        ([P0], [R - 1]),                                   # -P
        ([P0, P0, P0], [7, 7, 7]),                         # same bucket, doubling inside a bucket
        ([P0, bn.g1_neg(P0)], [5, 5]),                     # cancellation to infinity
        ([None, P1, None], [3, 4, 5]),                     # points at infinity
        ([P0, P1] * 40, [1] * 80),                         # one bucket gets every term
        ([P0, P1, P0], [2**128 + 1, 2**200 - 7, (R - 1) // 2]),
    ]
    for pts, sc in cases:
        got = nv.zkvc_msm_g1(_util.to_cuda(_util.g1_rows(pts)), _util.to_cuda(_util.ints_to_u8(sc)))
        assert got == bn.g1_bytes(bn.g1_msm(pts, sc)), (len(pts), sc[:3])


def test_msm_g1_full_size_closed_form(nv):
    """2^16 points with known discrete logs: the MSM must equal [sum s_i k_i] G."""
    rng = random.Random(77)
    n, block = 1 << 16, 1024
    pts, logs = [], []
    for _ in range(n // block):
        b, d = rng.randrange(1, R), rng.randrange(1, R)
        Pt, D = bn.g1_mul(bn.G1_GEN, b), bn.g1_mul(bn.G1_GEN, d)
        for i in range(block):
            pts.append(Pt)
            logs.append((b + i * d) % R)
            Pt = bn.g1_add(Pt, D)
    sc = [rng.randrange(R) for _ in range(n)]
    got = nv.zkvc_msm_g1(_util.to_cuda(_util.g1_rows(pts)), _util.to_cuda(_util.ints_to_u8(sc)))
    expect = bn.g1_mul(bn.G1_GEN, sum(s * k for s, k in zip(sc, logs)) % R)
    assert got == bn.g1_bytes(expect)


@pytest.mark.parametrize("n", [1, 5, 64, 300])
def test_msm_g2_random(nv, n):
    rng = random.Random(1000 + n)
    pts = [bn.g2_mul(bn.G2_GEN, rng.randrange(1, R)) for _ in range(n)]
    sc = [rng.randrange(R) for _ in range(n)]
    if n == 5:
        pts[1] = pts[0]
        sc[1] = sc[0]
        pts[3] = None
    got = nv.zkvc_msm_g2(_util.to_cuda(_util.g2_rows(pts)), _util.to_cuda(_util.ints_to_u8(sc)))
    assert got == bn.g2_bytes(bn.g2_msm(pts, sc))


def test_generator_mul(nv):
    rng = random.Random(31)
    sc = [0, 1, 2, bn.R - 1, (bn.R - 1) // 2] + [rng.randrange(bn.R) for _ in range(200)]
    t = _util.to_cuda(_util.ints_to_u8(sc))
    g1 = nv.zkvc_g1_generator_mul(t).cpu().numpy()
    assert bytes(g1.reshape(-1)) == b"".join(bn.g1_bytes(bn.g1_mul(bn.G1_GEN, k)) for k in sc)
    g2 = nv.zkvc_g2_generator_mul(t[:40]).cpu().numpy()
    assert bytes(g2.reshape(-1)) == b"".join(bn.g2_bytes(bn.g2_mul(bn.G2_GEN, k)) for k in sc[:40])
