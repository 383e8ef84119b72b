"""Parity at the sizes the benchmarks run, against the oracle.

* The one-proof benchmark's exact path at [49,320]x[320,512]: the key autotuned in the
  benchmark's mode (the tuner picks the prover mode and launch shape), fixed X, W, Y and
  workspace buffers so that zkvc_prove captures the proof on its second call and replays
  the captured CUDA graph after that, eight steps with the benchmark's (r, s) sequence;
  every proof equals the oracle's closed-form proof (tests/golden, written by
  tests/golden/make_closed_form.py from oracle/ alone).
* The kernel sweep's large sizes: G1 MSMs of 2^20 and 2^24 points and G2 MSMs of 2^16
  and 2^20 points with known discrete logs (points = [k_i] G made by the library's
  fixed-base kernel, spot-checked against the oracle's scalar multiplication), equal to
  [sum s_i k_i] G; NTTs of 2^24 points by round trips and sampled outputs evaluated one
  by one as polynomial values at powers of the root of unity.

* The largest sizes the library accepts: G1 and G2 MSMs of ZKVC_MSM_MAX_POINTS (2^27)
  points, tiled from 256 points of known discrete logs with uniform scalars, so that the
  expected [sum_j k_j t_j] G needs only the scalars' sums t_j over each tile class
  (exact byte-column sums on the device); and NTTs of 2^28 points (the domain's maximum):
  round trips of both kinds and the outputs at k = 0 and N/2 (the coefficients' sum and
  alternating sum).

All comparisons are exact."""
import os
import random

import numpy as np
import pytest

from oracle import bn254 as bn
from tests import _util

pytestmark = pytest.mark.gpu

R = bn.R
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def nv():
    import torch
    assert torch.cuda.is_available()
    return _util.native()


def _golden_cfg2():
    out = {}
    for line in open(os.path.join(GOLDEN, "closed_form_49x320x512.txt")):
        if line.startswith("#") or not line.strip():
            continue
        i, r, s, proof = line.split()
        out[int(i)] = (int(r, 16), int(s, 16), bytes.fromhex(proof))
    return out


def test_bench_path_replayed_graph_matches_oracle(nv):
    """bench.py's default workload, step for step: autotuned key, captured graph replays."""
    import torch

    from paper_2504_12217_gb300 import inputs
    a, n, b = inputs.SHAPE_CFG2
    seed = inputs.SEED_CFG[2]
    inst = inputs.instance(seed, (a, n, b))
    gold = _golden_cfg2()
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    Xd = torch.from_numpy(inst["X"]).cuda()
    Wd = torch.from_numpy(inst["W"]).cuda()
    Yd = torch.empty((a, b), dtype=torch.int32, device="cuda")
    nv.zkvc_pk_autotune(pk, Xd, Wd, inputs.to_bytes32(inst["rs"]), mode=nv.ZKVC_PROVE_AUTO)
    ws = torch.empty(nv.zkvc_prove_workspace_bytes(pk), dtype=torch.uint8, device="cuda")
    Yexp = inst["X"].astype(np.int64) @ inst["W"].astype(np.int64)
    for i in sorted(gold):
        r, s, expect = gold[i]
        assert (r, s) == tuple(inputs.prover_values(seed * 1000 + i))
        proof, _ = nv.zkvc_prove(pk, Xd, Wd, inputs.to_bytes32([r, s]), Y=Yd, workspace=ws)
        assert proof == expect, f"step {i} (tuning {nv.zkvc_pk_get_tuning(pk)})"
        assert np.array_equal(Yd.cpu().numpy(), Yexp), i
    assert nv.zkvc_verify(vk, inst["X"], Yexp.astype(np.int32), proof)


def _rand_scalars(gen, n):
    import torch
    t = torch.randint(0, 256, (n, 32), dtype=torch.uint8, generator=gen)
    t[:, 31] &= 0x0F  # below 2^252 < r: canonical
    return t


def _dot_mod_r(ka, sa):
    """sum_i k_i s_i mod r over two [n, 32] little-endian uint8 arrays."""
    rk, rs = ka.tobytes(), sa.tobytes()
    acc = 0
    fb = int.from_bytes
    for off in range(0, len(rk), 32):
        acc += fb(rk[off:off + 32], "little") * fb(rs[off:off + 32], "little")
    return acc % R


@pytest.mark.parametrize("group,log_n", [(1, 20), (1, 24), (2, 16), (2, 20)])
def test_msm_sweep_sizes_known_logs(nv, group, log_n):
    import torch
    n = 1 << log_n
    gen = torch.Generator().manual_seed(9000 + 100 * group + log_n)
    k = _rand_scalars(gen, n)
    s = _rand_scalars(gen, n)
    s[1] = 0  # zero scalar
    kd = k.cuda()
    pts = nv.zkvc_g1_generator_mul(kd) if group == 1 else nv.zkvc_g2_generator_mul(kd)
    del kd
    rng = random.Random(log_n)
    mul, enc, width = (bn.g1_mul, bn.g1_bytes, 64) if group == 1 else (bn.g2_mul, bn.g2_bytes, 128)
    gen_pt = bn.G1_GEN if group == 1 else bn.G2_GEN
    kn = k.numpy()
    for i in [0, n - 1] + [rng.randrange(n) for _ in range(6)]:
        ki = int.from_bytes(kn[i].tobytes(), "little")
        assert bytes(pts[i].cpu().numpy()) == enc(mul(gen_pt, ki)), i
    sd = s.cuda()
    ws = torch.empty(nv.zkvc_msm_workspace_bytes(n, group), dtype=torch.uint8, device="cuda")
    got = nv.zkvc_msm_g1(pts, sd, ws) if group == 1 else nv.zkvc_msm_g2(pts, sd, ws)
    assert len(got) == width
    assert got == enc(mul(gen_pt, _dot_mod_r(kn, s.numpy())))
    del pts, sd, ws
    torch.cuda.empty_cache()


def _poly_at(coeffs_u8, x):
    """sum_i a_i x^i mod r (Horner) over [n, 32] little-endian uint8 coefficients."""
    raw = coeffs_u8.tobytes()
    acc = 0
    fb = int.from_bytes
    for off in range(len(raw) - 32, -32, -32):
        acc = (acc * x + fb(raw[off:off + 32], "little")) % R
    return acc


def test_ntt_2_24(nv):
    """2^24 points: forward/inverse and coset round trips; forward outputs at k = 0,
    N/2 (sums with signs), 1 and a random k, and one coset-forward output, each the
    input polynomial evaluated at omega^k (g omega^k for the coset)."""
    import torch
    log_n = 24
    n = 1 << log_n
    gen = torch.Generator().manual_seed(24)
    raw = _rand_scalars(gen, n)
    x = raw.cuda()
    t = x.clone()
    nv.zkvc_ntt(t, 2)
    nv.zkvc_ntt(t, 3)
    assert torch.equal(t, x)
    t.copy_(x)
    nv.zkvc_ntt(t, 0)
    out = t.cpu().numpy()
    a = raw.numpy()
    w = bn.fr_root_of_unity(n)
    ks = [0, n // 2, 1, random.Random(7).randrange(n)]
    for k in ks:
        assert int.from_bytes(out[k].tobytes(), "little") == _poly_at(a, pow(w, k, R)), k
    nv.zkvc_ntt(t, 1)
    assert torch.equal(t, x)
    t.copy_(x)
    nv.zkvc_ntt(t, 2)
    k = 12345
    assert int.from_bytes(t[k].cpu().numpy().tobytes(), "little") == _poly_at(a, 5 * pow(w, k, R) % R)
    del t, x
    torch.cuda.empty_cache()


def _class_sums(s_u8, classes):
    """[sum of s_i over i = j mod classes for j < classes] as integers: exact, from int64
    sums of each byte column on the device."""
    import torch
    n = s_u8.shape[0]
    cols = s_u8.view(n // classes, classes, 32).sum(dim=0, dtype=torch.int64).cpu().tolist()
    return [sum(v << (8 * b) for b, v in enumerate(row)) for row in cols]


@pytest.mark.parametrize("group", [1, 2])
def test_msm_max_size(nv, group):
    import torch
    n, classes = nv.ZKVC_MSM_MAX_POINTS, 256
    rng = random.Random(4242 + group)
    if group == 1:
        mul, enc, rows, call, gen_pt = bn.g1_mul, bn.g1_bytes, _util.g1_rows, nv.zkvc_msm_g1, bn.G1_GEN
    else:
        mul, enc, rows, call, gen_pt = bn.g2_mul, bn.g2_bytes, _util.g2_rows, nv.zkvc_msm_g2, bn.G2_GEN
    logs = [rng.randrange(1, R) for _ in range(classes)]
    tile = torch.from_numpy(rows([mul(gen_pt, k) for k in logs])).cuda()
    pts = tile.repeat(n // classes, 1)  # point i = [logs[i mod classes]] G
    del tile
    g = torch.Generator(device="cuda").manual_seed(0x5A4B0000 + group)
    s = torch.randint(0, 256, (n, 32), dtype=torch.uint8, device="cuda", generator=g)
    s[:, 31] &= 0x0F
    s[7] = 0
    ws = torch.empty(nv.zkvc_msm_workspace_bytes(n, group), dtype=torch.uint8, device="cuda")
    got = call(pts, s, ws)
    del pts, ws
    torch.cuda.empty_cache()
    sums = _class_sums(s, classes)
    assert got == enc(mul(gen_pt, sum(k * t for k, t in zip(logs, sums)) % R))
    del s
    torch.cuda.empty_cache()


def test_ntt_max_size_2_28(nv):
    import torch
    n = 1 << 28
    g = torch.Generator(device="cuda").manual_seed(28)
    x = torch.randint(0, 256, (n, 32), dtype=torch.uint8, device="cuda", generator=g)
    x[:, 31] &= 0x0F
    even, odd = _class_sums(x, 2)
    t = x.clone()
    nv.zkvc_ntt(t, 0)
    assert int.from_bytes(t[0].cpu().numpy().tobytes(), "little") == (even + odd) % R
    assert int.from_bytes(t[n // 2].cpu().numpy().tobytes(), "little") == (even - odd) % R
    nv.zkvc_ntt(t, 1)
    assert torch.equal(t, x)
    nv.zkvc_ntt(t, 2)
    nv.zkvc_ntt(t, 3)
    assert torch.equal(t, x)
    del t, x
    torch.cuda.empty_cache()
