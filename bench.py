"""Benchmark: CRPC-matmul Groth16 proofs/s (BN254) with p50/p99 latency on GB300.

Workload: one Groth16 proof of the CRPC + PSQ circuit for Y = X W with X int8 [49, 320]
and W int8 [320, 512] (entries uniform in [-128, 127], seeded SplitMix64; setup toxic
waste and prover (r, s) seeded the same way).  A step is one full prove: witness, CRPC
and PSQ evaluation, the NTT chain to h(x), every MSM, and the proof encoding.

* ``value``   proofs/s over the timed steps, inputs resident in HBM (device-timed with
              CUDA events on the prover's stream; L2 flushed by a 256 MiB write between
              steps, outside the events).
* ``e2e``     the same metric through the public API with pinned host inputs: every
              step copies X and W host->device and reads Y and the proof back.
* ``roofline`` the bucket accumulation of the H-query MSM (the G1 run with the most
              algorithmic work), timed live with CUDA events on its stream; its algorithmic
              work is one mixed point addition per bucket term (10 Montgomery products of
              264 32-bit IMADs in G1).
* ``ntt_roofline`` the prover's NTT chain live at 2^16 points and one 2^24-point
              transform: fractions of the measured integer peak and of HBM bandwidth.
* ``batched`` / ``served`` the 64-proof batched workload (one captured graph per 64
              proofs) and Poisson-served requests over 32 shapes, each beside the plain
              one-proof path on the same instances.
* ``cpu_baseline`` the oracle (tests' reference implementation) proving one whole
              instance on all host cores, measured.

With ``--gpus N`` under torchrun every rank proves its own instances (replicas: proofs
are independent, no collective on the data path); value = all proofs / max rank time.
``--impl reference`` times the oracle instead (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CRPC-matmul Groth16 proofs/s + p50/p99 latency; MSM/NTT % of roofline"
UNIT = "proofs/s"
SHAPE = (49, 320, 512)
IMAD_PER_CLK_SM = 64          # nominal 32-bit integer multiply-add rate per SM per clock (context)
MONT_IMAD = 4 * 8 * 8 + 8     # CIOS product on 8 x 32-bit limbs
G1_MADD_PRODUCTS = 10         # madd-2008-s: 8M + 2S
G2_MADD_PRODUCTS = 30         # the same over Fp2, 3 Fp products per Fp2 product


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ------------------------------------------------------------------ replicas
def rank_seed(base, rank):
    """Seed of the instances rank `rank` proves: ranks are replicas over disjoint inputs
    (proofs are independent, so no collective touches the data path)."""
    return base + 7919 * rank


def reduce_max(x, dist, device):
    """Max over ranks of a host float (the timed region's length); identity without dist."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, world, seconds_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle baseline
# The oracle (the tests' plain reference implementation) proving one [49,320]x[320,512]
# instance on the host cores: the steps of oracle.groth16.prove -- witness, domain
# evaluations, the quotient through the textbook NTTs, every naive MSM -- with the
# independent transforms and the MSMs' point ranges spread over a spawn pool of worker
# processes (one per core).  Proving-key points stand in as arithmetic progressions
# [c + i d]G of the right counts (the oracle's own setup at this size would take about
# 40 core-minutes, and an MSM's cost does not depend on which points it sums).

def _oracle_points(job):
    """Stand-in key points: [c + i d] G for i < count, by repeated affine addition."""
    from oracle import bn254 as bn
    group, c, d, count = job
    mul, add, gen = (bn.g1_mul, bn.g1_add, bn.G1_GEN) if group == 1 else (bn.g2_mul, bn.g2_add, bn.G2_GEN)
    P, D = mul(gen, c), mul(gen, d)
    out = []
    for _ in range(count):
        out.append(P)
        P = add(P, D)
    return out


def _oracle_task(job):
    """One unit of the oracle's prove: a transform of oracle.ntt, or a naive MSM slice."""
    from oracle import bn254 as bn
    from oracle import ntt as nt
    kind = job[0]
    if kind == "ntt":
        return getattr(nt, job[1])(job[2])
    pts, sc = job[1], job[2]
    return bn.g1_msm(pts, sc) if kind == "g1" else bn.g2_msm(pts, sc)


class OracleProver:
    """Key stand-ins and the pool, made once (not timed); prove() times one proof."""

    def __init__(self, seed, cores=None):
        import multiprocessing as mp
        import random

        from oracle import crpc
        from paper_2504_12217_gb300 import inputs
        a, n, b = SHAPE
        self.inst = inputs.instance(seed, SHAPE)
        self.z = self.inst["toxic"][5]
        self.shape = crpc.Shape(a, n, b)
        self.rows = crpc.build_r1cs(self.shape, self.z)
        sA, sB = set(), set()
        for A, B, _ in self.rows:
            sA.update(A)
            sB.update(B)
        self.A_vars, self.B_vars = sorted(sA), sorted(sB)
        self.L_vars = list(range(self.shape.n_public + 1, self.shape.n_vars))
        self.N = self.shape.domain
        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        rng = random.Random(seed)
        counts = {"A": len(self.A_vars), "B1": len(self.B_vars), "L": len(self.L_vars), "H": self.N - 1}
        self.pts = {}
        for name, cnt in list(counts.items()) + [("B2", len(self.B_vars))]:
            group = 2 if name == "B2" else 1
            step = max(1, cnt // (4 * self.cores) + 1)
            jobs = [(group, rng.randrange(1, 1 << 250), rng.randrange(1, 1 << 250), min(step, cnt - o))
                    for o in range(0, cnt, step)]
            self.pts[name] = [p for part in self.pool.map(_oracle_points, jobs) for p in part]
        self.consts = _oracle_points((1, rng.randrange(1, 1 << 250), 1, 4)) + _oracle_points(
            (2, rng.randrange(1, 1 << 250), 1, 2))

    def close(self):
        self.pool.terminate()

    def prove(self, r, s, frac=1.0):
        """Seconds of one proof; frac < 1 runs each MSM on that share of its terms and
        scales its part by the term counts (the witness and quotient always run whole)."""
        from oracle import bn254 as bn
        from oracle import crpc
        from oracle import groth16 as og
        X = self.inst["X"].astype(int).tolist()
        W = self.inst["W"].astype(int).tolist()
        N = self.N
        parts = {}
        t0 = time.perf_counter()
        Y = crpc.matmul_int(X, W)
        w = crpc.witness(self.shape, X, W, self.z, Y)
        Aev, Bev, Cev = og.domain_evaluations(self.rows, w, N)
        parts["witness"] = time.perf_counter() - t0
        t1 = time.perf_counter()
        a, b, c = self.pool.map(_oracle_task, [("ntt", "intt", v) for v in (Aev, Bev, Cev)])
        ae, be, ce = self.pool.map(_oracle_task, [("ntt", "coset_ntt", v) for v in (a, b, c)])
        zinv = pow((pow(bn.FR_GEN, N, bn.R) - 1) % bn.R, -1, bn.R)
        hev = [((x * y - zz) * zinv) % bn.R for x, y, zz in zip(ae, be, ce)]
        h = self.pool.apply(_oracle_task, (("ntt", "coset_intt", hev),))
        parts["quotient"] = time.perf_counter() - t1
        t2 = time.perf_counter()
        msms = [("g1", "A", [w[i] for i in self.A_vars]), ("g1", "B1", [w[i] for i in self.B_vars]),
                ("g2", "B2", [w[i] for i in self.B_vars]), ("g1", "L", [w[i] for i in self.L_vars]),
                ("g1", "H", h[:N - 1])]
        jobs, owner, scale = [], [], {}
        for kind, name, sc in msms:
            pts = self.pts[name]
            take = max(1, int(len(sc) * frac))
            scale[name] = len(sc) / take
            step = max(1, take // (4 * self.cores) + 1)
            for o in range(0, take, step):
                jobs.append((kind, pts[o:o + step], sc[o:o + step]))
                owner.append(name)
        order = sorted(range(len(jobs)), key=lambda j: owner[j] != "H")
        res = self.pool.map(_oracle_task, [jobs[j] for j in order], chunksize=1)
        sums = {}
        for j, v in zip(order, res):
            nm = owner[j]
            sums[nm] = (bn.g2_add if nm == "B2" else bn.g1_add)(sums.get(nm), v)
        al, be1, de1, _, be2, de2 = self.consts
        A = bn.g1_add(bn.g1_add(al, sums["A"]), bn.g1_mul(de1, r))
        B1 = bn.g1_add(bn.g1_add(be1, sums["B1"]), bn.g1_mul(de1, s))
        bn.g2_add(bn.g2_add(be2, sums["B2"]), bn.g2_mul(de2, s))
        C = bn.g1_add(sums["L"], sums["H"])
        C = bn.g1_add(C, bn.g1_mul(A, s))
        C = bn.g1_add(C, bn.g1_mul(B1, r))
        bn.g1_add(C, bn.g1_neg(bn.g1_mul(de1, r * s % bn.R)))
        msm_s = time.perf_counter() - t2
        parts["msm"] = msm_s * (max(scale.values()) if frac < 1.0 else 1.0)
        total = parts["witness"] + parts["quotient"] + parts["msm"]
        return total, parts


def cpu_baseline(args):
    """One whole oracle proof of the benchmark's instance on all host cores (measured)."""
    from paper_2504_12217_gb300 import inputs
    seed = inputs.SEED_CFG[2]
    t0 = time.perf_counter()
    op = OracleProver(seed)
    prep = time.perf_counter() - t0
    try:
        r, s = inputs.prover_values(seed)
        sec, parts = op.prove(r, s)
    finally:
        op.close()
    return {"value": 1.0 / sec, "unit": UNIT, "cores": op.cores, "kind": "oracle",
            "sample": "one whole [49,320]x[320,512] proof with the oracle's prove steps (witness, domain "
                      "evaluations, textbook-NTT quotient, every naive MSM), transforms and MSM point ranges "
                      "over a spawn pool of all host cores; key points are stand-in arithmetic progressions "
                      "of the right counts (built before timing)",
            "seconds_per_proof": sec, "parts_s": parts, "key_standins_s": prep}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    from paper_2504_12217_gb300 import inputs
    seed = inputs.SEED_CFG[2]
    frac = 1.0 / 16
    op = OracleProver(seed)
    try:
        total = args.warmup + args.steps
        rs = [inputs.prover_values(seed * 1000 + i) for i in range(total)]
        for i in range(args.warmup):
            op.prove(*rs[i], frac=frac)
        times = []
        t0 = time.perf_counter()
        for i in range(args.steps):
            sec, _ = op.prove(*rs[args.warmup + i], frac=frac)
            times.append(sec)
        wall = time.perf_counter() - t0
    finally:
        op.close()
    per_proof = statistics.median(times)
    value = 1.0 / per_proof
    sample = ("per step: the oracle's prove steps for the [49,320]x[320,512] instance on a spawn pool of all host "
              "cores -- witness, domain evaluations and the textbook-NTT quotient whole, each naive MSM on 1/16 "
              "of its terms with its time scaled by 16; key points are stand-in arithmetic progressions")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_proof * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "python-int (exact)", "data": "synthetic",
        "config": {"workload": "crpc_groth16_bn254_49x320x512", "a": SHAPE[0], "n": SHAPE[1], "b": SHAPE[2],
                   "log_domain": 16},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": op.cores, "kind": "oracle", "sample": sample,
                         "extrapolated": True, "wall_s": wall,
                         "note": "ms_per_step is the extrapolated time of one whole proof; the timed steps "
                                 "themselves ran the sample above"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ kernel sweep
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def nominal_imad_peak(sms, mhz):
    """The unit-count figure the measured peak stands beside: SMs x 64 IMAD/clk x clock."""
    return sms * IMAD_PER_CLK_SM * mhz * 1e6


def measure_imad_peak(nv, local):
    """The integer-pipe peak measured on this GPU (zkvc_imad_rate): the fastest of the
    microbenchmark forms (a 32 x 32 -> 64-bit product counted as two IMADs, as in the 264
    of a Montgomery product), with the SM clock sampled while it runs."""
    clocks = ClockSampler(local)
    clocks.start()
    names = ("independent_mad_lo", "cios_carry_row", "independent_mad_hi", "independent_mad_wide",
             "mad_lo_carry_chains")
    forms = {name: nv.zkvc_imad_rate(f, 1 << 18) for f, name in enumerate(names)}
    # whole Montgomery products (reported beside the peak, not candidates for it)
    products = {"fp_mul_carry_chain": nv.zkvc_imad_rate(5, 1 << 11), "fp_mulc_64bit_acc": nv.zkvc_imad_rate(6, 1 << 11)}
    clk = clocks.stop()
    best = max(forms.values(), key=lambda f: f["imad_per_s"])
    return {"imad_per_s": best["imad_per_s"], "sms": best["sms"], "forms": forms, "montgomery_products": products,
            "clocks": clk}


def ntt_passes(log_n):
    """HBM passes of one transform as the method counts them: one below 2^20 points
    (the transform fits on chip per block of stages), two from 2^20 up."""
    return 1 if log_n < 20 else 2


def ntt_work(log_n, transforms=1):
    """(IMADs, bytes) of `transforms` radix-2 NTTs of 2^log_n points: (N/2) log N
    butterflies of one Montgomery product each, and 64 B per point per HBM pass."""
    n = 1 << log_n
    return transforms * (n // 2) * log_n * MONT_IMAD, transforms * ntt_passes(log_n) * 64 * n


def ntt_roofline(nv, prof, log_n_proof, imad_peak, hbm_peak, hbm_src):
    """NTT fractions of the integer and HBM peaks: the quotient chain live in the proof
    (seven transforms of 2^16 points and the pointwise quotient), and one timed 2^24
    forward transform on uniform Fr data."""
    import torch
    out = {"bytes_rule": "64 B per point per HBM pass; 1 pass below 2^20 points, 2 from 2^20",
           "imad_rule": "(N/2) log2 N butterflies x 264 IMAD per transform (scalings and the quotient's "
                        "products not counted)"}
    st = prof.get("ntt", {"ms": 0, "calls": 0})
    if st["calls"]:
        ms = st["ms"] / st["calls"]
        imad, nbytes = ntt_work(log_n_proof, 7)
        out["in_proof"] = {"log_n": log_n_proof, "transforms": 7, "ms": ms,
                           "imad_frac": imad / (ms / 1e3) / imad_peak, "hbm_gbs": nbytes / ms / 1e6,
                           "hbm_frac": nbytes / ms / 1e6 / hbm_peak,
                           "note": "the prover's quotient chain (3 INTT, 3 coset NTT, quotient, coset INTT) on "
                                   "its stream, stage timers"}
    log_n = 24
    n = 1 << log_n
    g = torch.Generator(device="cuda").manual_seed(0x5A4B5643_00000003)
    x = torch.randint(0, 256, (n, 32), dtype=torch.uint8, device="cuda", generator=g)
    x[:, 31] &= 0x0F
    nv.zkvc_ntt(x, 0)
    torch.cuda.synchronize()
    reps = 5
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in evs:  # 512 MiB of points: larger than L2 on its own
        e0.record()
        nv.zkvc_ntt(x, 0)
        e1.record()
    torch.cuda.synchronize()
    ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in evs)
    imad, nbytes = ntt_work(log_n)
    out["full_2e24"] = {"log_n": log_n, "kind": "forward", "ms": ms, "imad_frac": imad / (ms / 1e3) / imad_peak,
                        "hbm_gbs": nbytes / ms / 1e6, "hbm_frac": nbytes / ms / 1e6 / hbm_peak}
    out["hbm_peak_gbs"] = hbm_peak
    out["hbm_peak_source"] = hbm_src
    out["imad_peak_tops"] = imad_peak / 1e12
    del x
    torch.cuda.empty_cache()
    return out


def msm_work(group, logn):
    """IMAD-equivalents of the library's variable-base MSM of 2^logn points, and its window
    bits c (window rule: log2(points) - 3 within [4, 16], then the smallest c with the
    same window count).  Both groups run an endomorphism split (G1: GLV with phi, G2:
    psi): 2N points of 127-bit scalars, 2N ceil(128/c) mixed additions and 2^c
    ceil(128/c) full additions for the bucket sums."""
    pts_log, bits = logn + 1, 128
    win = -(-bits // min(16, max(4, pts_log - 3)))
    c = -(-bits // win)
    madd = G1_MADD_PRODUCTS if group == 1 else G2_MADD_PRODUCTS
    add = 14 if group == 1 else 42
    return ((1 << pts_log) * win * madd + (1 << c) * win * add) * MONT_IMAD, c


def msm_sweep_section(nv, imad_peak, local=0):
    """Variable-base MSMs of the kernel sweep inside the default line: G1 at 2^20 and 2^24
    points, G2 at 2^20, uniform Fr scalars, points = generator x uniform scalars (made by
    the library's fixed-base kernel, untimed).  Fractions of the integer peak with the
    method's work (msm_work).  Each call is timed on its own (CUDA events); `ms` is the
    median call, with every call's time and the SM clocks sampled meanwhile beside it."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(0x5A4B5643_00000003)

    def rand_fr(n):
        t = torch.randint(0, 256, (n, 32), dtype=torch.uint8, device="cuda", generator=g)
        t[:, 31] &= 0x0F
        return t

    out = []
    for group, logn in ((1, 20), (1, 24), (2, 20)):
        n = 1 << logn
        k = rand_fr(n)
        pts = nv.zkvc_g1_generator_mul(k) if group == 1 else nv.zkvc_g2_generator_mul(k)
        del k
        sc = rand_fr(n)
        ws = torch.empty(nv.zkvc_msm_workspace_bytes(n, group), dtype=torch.uint8, device="cuda")
        fn = (lambda: nv.zkvc_msm_g1(pts, sc, ws)) if group == 1 else (lambda: nv.zkvc_msm_g2(pts, sc, ws))
        fn()
        torch.cuda.synchronize()
        reps = 3
        clocks = ClockSampler(local)
        clocks.start()
        calls = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            calls.append(e0.elapsed_time(e1))
        clk = clocks.stop()
        ms = statistics.median(calls)
        work, c = msm_work(group, logn)
        point = {"group": f"G{group}", "log_n": logn, "ms": ms, "calls_ms": calls, "mpoints_per_s": n / ms / 1e3,
                 "imad_frac": work / (ms / 1e3) / imad_peak, "window_bits": c, "clocks": clk}
        if (group, logn) in MSM_ACCUM_TRAFFIC:
            terms = (2 * n) * -(-128 // c)
            point["accum_traffic"] = {"dram_bytes": MSM_ACCUM_TRAFFIC[(group, logn)],
                                      "algorithmic_bytes": terms * (64 * group + 4),
                                      "source": "one ncu capture of the accumulation launch at this size"}
        out.append(point)
        del pts, sc, ws
        torch.cuda.empty_cache()
    return {"msms": out, "note": "each call synchronises and reads its result back (zkvc_msm_g1/g2); "
                                  "inputs larger than L2 at 2^24 (1.5 GB)"}


def run_sweep(args):
    """NTT / INTT / coset NTT at 2^16..2^24 and G1 (2^16..2^24) / G2 (2^16..2^20) MSMs on
    uniform random Fr data, points = generator x seeded random scalars.  One JSON line."""
    import torch

    from paper_2504_12217_gb300 import native as nv

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    hbm, hbm_src = _peaks()
    imad = measure_imad_peak(nv, _env_int("LOCAL_RANK", 0))
    imad_peak = imad["imad_per_s"]
    g = torch.Generator(device="cuda").manual_seed(0x5A4B5643_00000003)

    def rand_fr(n):
        t = torch.randint(0, 256, (n, 32), dtype=torch.uint8, device="cuda", generator=g)
        t[:, 31] &= 0x0F
        return t

    def time_it(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"ntt": [], "msm_g1": [], "msm_g2": []}
    for logn in args.sweep_ntt:
        n = 1 << logn
        x = rand_fr(n)
        for kind, name in ((0, "ntt"), (1, "intt"), (2, "coset_ntt")):
            ms = time_it(lambda: nv.zkvc_ntt(x, kind), 5)
            work, bytes_moved = ntt_work(logn)
            out["ntt"].append({"log_n": logn, "kind": name, "ms": ms,
                               "hbm_gbs": bytes_moved / ms / 1e6, "hbm_frac": bytes_moved / ms / 1e6 / hbm,
                               "imad_frac": work / (ms / 1e3) / imad_peak})
        del x
        torch.cuda.empty_cache()
    for group, sizes in ((1, args.sweep_g1), (2, args.sweep_g2)):
        key = "msm_g1" if group == 1 else "msm_g2"
        for logn in sizes:
            n = 1 << logn
            k = rand_fr(n)
            pts = nv.zkvc_g1_generator_mul(k) if group == 1 else nv.zkvc_g2_generator_mul(k)
            del k
            sc = rand_fr(n)
            ws = torch.empty(nv.zkvc_msm_workspace_bytes(n, group), dtype=torch.uint8, device="cuda")
            fn = (lambda: nv.zkvc_msm_g1(pts, sc, ws)) if group == 1 else (lambda: nv.zkvc_msm_g2(pts, sc, ws))
            ms = time_it(fn, 3 if logn < 22 else 1)
            work, c = msm_work(group, logn)
            out[key].append({"log_n": logn, "ms": ms, "mpoints_per_s": n / ms / 1e3,
                             "imad_frac": work / (ms / 1e3) / imad_peak, "window_bits": c})
            del pts, sc, ws
            torch.cuda.empty_cache()
    line = {"metric": "kernel sweep: NTT/INTT/coset-NTT and G1/G2 MSM over BN254", "unit": "ms",
            "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src, "imad_peak_tops": imad_peak / 1e12,
            "imad_peak_source": "measured (zkvc_imad_rate)", "imad_microbenchmark": imad,
            "ntt_bytes_rule": "64 B per point per HBM pass; 1 pass below 2^20 points, 2 from 2^20",
            "data": "synthetic (uniform Fr; points = generator x random scalars)", "sweep": out}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def p99_of(xs):
    srt = sorted(xs)
    return srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]


def run_gpu(args):
    import torch

    from paper_2504_12217_gb300 import inputs
    from paper_2504_12217_gb300 import native as nv

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    a, n, b = SHAPE
    seed = rank_seed(inputs.SEED_CFG[2], rank)
    inst = inputs.instance(seed, SHAPE)
    pk, vk = nv.zkvc_setup(a, n, b, inputs.to_bytes32(inst["toxic"]))
    Xd = torch.from_numpy(inst["X"]).cuda()
    Wd = torch.from_numpy(inst["W"]).cuda()
    Yd = torch.empty((a, b), dtype=torch.int32, device="cuda")
    # one-time latency tuning of the key's launch shape (setup, not timed)
    if args.key_tuning:
        nv.zkvc_pk_set_tuning(pk, args.key_tuning)
        tuning = nv.zkvc_pk_get_tuning(pk)
    elif args.no_autotune:
        tuning = nv.zkvc_pk_get_tuning(pk)
    else:
        tuning = nv.zkvc_pk_autotune(pk, Xd, Wd, inputs.to_bytes32(inst["rs"]), mode=nv.ZKVC_PROVE_AUTO)
    ws = torch.empty(nv.zkvc_prove_workspace_bytes(pk), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    total_steps = args.warmup + args.steps
    rs_list = [inputs.to_bytes32(inputs.prover_values(seed * 1000 + i)) for i in range(total_steps)]

    for i in range(args.warmup):
        nv.zkvc_prove(pk, Xd, Wd, rs_list[i], Y=Yd, workspace=ws)
    torch.cuda.synchronize()

    # ---- device-timed steps, inputs resident (zkvc_prove replays its captured graph)
    launches0 = nv.zkvc_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record()
        nv.zkvc_prove(pk, Xd, Wd, rs_list[args.warmup + i], Y=Yd, workspace=ws)
        evs[i][1].record()
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    launches = nv.zkvc_kernel_launches() - launches0
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_s = reduce_max(sum(step_ms) / 1e3, dist, "cuda")
    value = replica_value(args.steps, world, total_s)

    # ---- end to end through the public API: pinned host inputs, results read back
    Xh = torch.from_numpy(inst["X"]).pin_memory()
    Wh = torch.from_numpy(inst["W"]).pin_memory()
    Yh = torch.empty((a, b), dtype=torch.int32).pin_memory()
    e2e_steps = max(3, args.steps)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        Xd.copy_(Xh, non_blocking=True)
        Wd.copy_(Wh, non_blocking=True)
        proof, _ = nv.zkvc_prove(pk, Xd, Wd, rs_list[i % total_steps], Y=Yd, workspace=ws)
        Yh.copy_(Yd, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": replica_value(e2e_steps, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": a * n + n * b,
           "d2h_bytes_per_step": 256 + 4 * a * b}

    # ---- stage timers (events on the prover's streams; zkvc_prove enqueues directly while
    # they are on): the accumulation kernels' live durations for the roofline and the
    # proof's timeline across its streams
    nv.zkvc_profile_enable(True)
    for i in range(min(args.steps, 50)):
        flush.zero_()
        nv.zkvc_prove(pk, Xd, Wd, rs_list[args.warmup + i], Y=Yd, workspace=ws)
    torch.cuda.synchronize()
    prof = nv.zkvc_profile_read()
    nv.zkvc_profile_enable(False)
    del flush
    torch.cuda.empty_cache()

    # ---- the integer-pipe peak of this GPU (microbenchmark, outside the timed region)
    imad = measure_imad_peak(nv, local)
    peak = imad["imad_per_s"] / 1e12
    hbm, hbm_src = _peaks()

    # ---- the batched and served forms beside the plain one-proof path (1 GPU, rank 0)
    batched = served = None
    if world == 1 and not args.no_batched:
        batched = batched_section(nv, args, local)
    if world == 1 and not args.no_served:
        served = served_section(nv, args, local)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (bucket accumulation), timed live
    g1 = prof.get("msm_g1_bucket_accum", {"ms": 0, "units": 0, "calls": 0})
    g2 = prof.get("msm_g2_bucket_accum", {"ms": 0, "units": 0, "calls": 0})
    w1 = g1["units"] * G1_MADD_PRODUCTS * MONT_IMAD
    w2 = g2["units"] * G2_MADD_PRODUCTS * MONT_IMAD
    # the dominant kernel is the accumulation with the most algorithmic work: the H-query
    # run in G1 (its time share also leads the launch list)
    dom, work, ms, calls = ("k_accum0<G1> (H query)", w1, g1["ms"], g1["calls"]) if w1 >= w2 else \
        ("k_accum0<G2>", w2, g2["ms"], g2["calls"])
    achieved = (work / calls) / (ms / calls / 1e3) / 1e12 if ms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TIMAD/s",
                "frac": achieved / peak, "traffic": H_ACCUM_TRAFFIC.get(tuning[2]) if dom.startswith("k_accum0<G1>")
                else None, "traffic_unit": "bytes per launch",
                "peak_source": "measured on this GPU by zkvc_imad_rate (of measured), the fastest of five "
                               "multiply-add forms",
                "peak_nominal": nominal_imad_peak(imad["sms"], 2070.0) / 1e12,
                "algorithmic_imad_per_launch": work / max(calls, 1),
                "launch_ms": ms / max(calls, 1)}
    stages = {k: round(v["ms"] / max(v["calls"], 1), 4) for k, v in prof.items()}
    spans = {k: [round(v["start_ms"], 4), round(v["end_ms"], 4)] for k, v in prof.items() if v["calls"]}
    nttr = ntt_roofline(nv, prof, 16, imad["imad_per_s"], hbm, hbm_src)
    msweep = msm_sweep_section(nv, imad["imad_per_s"], local) if not args.no_msm_sweep else None

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    srt = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 limbs (exact Fr/Fp arithmetic)",
        "data": "synthetic",
        "config": {"workload": "crpc_groth16_bn254_49x320x512", "a": a, "n": n, "b": b, "log_domain": 16,
                   "l2": "flushed by a 256 MiB write between steps", "parallelism": f"replicas x{world}",
                   "msm_chunks_small_rest_h_g2": tuning[:4], "ntt_log_elems_per_block": tuning[4] or 10,
                   "side_msm_start": ("at once", "after the NTTs", "after the H accumulation")[tuning[5]],
                   "prover_mode": ("fold", "chain")[tuning[6]],
                   "g2_msm_start": ("at once", "after the NTTs")[tuning[7]],
                   "quad_lanes_h_small": tuning[8:10],
                   "chunk_source": "imposed (--key-tuning)" if args.key_tuning else
                   "default rule" if args.no_autotune else "zkvc_pk_autotune at setup"},
        "latency_ms": {"p50": statistics.median(step_ms), "p99": p99_of(step_ms), "min": srt[0], "max": srt[-1]},
        "e2e": e2e, "roofline": roofline, "ntt_roofline": nttr, "msm_sweep": msweep, "imad_peak": imad,
        "batched": batched, "served": served, "cpu_baseline": cpu, "gpu_launches": launches,
        "gpu_launches_per_step": launches / args.steps, "clocks": clk, "stage_ms": stages,
        "stage_span_ms": spans,
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# DRAM bytes (read + write) of one H-query accumulation launch of the [49,320]x[320,512]
# proof, from one ncu capture of the balanced accumulation (product-scanning products)
# with the default chunk rule, which gives this run 16 terms per chunk, so an imposed
# chunk of 16 is the same launch (dram__bytes_read.sum + dram__bytes_write.sum); other
# chunk settings: not captured
H_ACCUM_TRAFFIC = {0: 76589568, 16: 76589568}

# DRAM bytes (read + write) of the accumulation launch of the variable-base MSMs of the
# sweep points, from one ncu capture per size (dram__bytes_read.sum +
# dram__bytes_write.sum), beside the launch's algorithmic bytes: one 64-byte base and one
# 4-byte sorted index per bucket term (2^(log_n + 1) split points x 8 windows)
MSM_ACCUM_TRAFFIC = {(1, 20): 1104113000 + 41336576}


# ------------------------------------------------------------------ batched workload
def shape_seed(base, shape):
    a, n, b = shape
    return base ^ (a << 40) ^ (n << 20) ^ b


def batched_setup(nv, inputs, shapes):
    """One proving key per distinct shape of the mix (setup seeds by shape)."""
    keys, vkeys = {}, {}
    for s in dict.fromkeys(shapes):
        keys[s], vkeys[s] = nv.zkvc_setup(*s, inputs.to_bytes32(inputs.setup_values(shape_seed(inputs.SEED_CFG[4], s))))
    return keys, vkeys


def batched_core(nv, shapes, keys, steps, warmup, local, tuning=None, eager=False, autotune=True):
    """Times `steps` calls of one batched prove over `shapes` (one instance each) after
    autotuning and capture: device time per call with CUDA events, L2 flushed between
    calls.  Returns a dict of measurements plus the objects the callers reuse."""
    import torch

    from paper_2504_12217_gb300 import inputs
    sets = []
    for v in range(2):
        insts = [inputs.instance(inputs.SEED_CFG[4] + 1000 * (v + 1) + i, s) for i, s in enumerate(shapes)]
        sets.append(([torch.from_numpy(t["X"]).cuda() for t in insts], [torch.from_numpy(t["W"]).cuda() for t in insts],
                     [inputs.to_bytes32(t["rs"]) for t in insts], insts))
    Ys = [torch.empty((s[0], s[2]), dtype=torch.int32, device="cuda") for s in shapes]
    t0 = time.perf_counter()
    flags = nv.ZKVC_BATCH_EAGER if eager else 0
    if autotune and not tuning:
        flags |= nv.ZKVC_BATCH_AUTOTUNE
    batch = nv.Batch([keys[s] for s in shapes], flags=flags)
    if tuning:
        batch.set_tuning(tuning)
    nv.zkvc_set_wait_timeout_ms(120000)
    batch.prove(sets[0][0], sets[0][1], sets[0][2], Ys)  # autotune + capture
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    for i in range(warmup):
        x = sets[i % 2]
        batch.prove(x[0], x[1], x[2], Ys)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = nv.zkvc_kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        x = sets[i % 2]
        flush.zero_()
        evs[i][0].record()
        batch.prove(x[0], x[1], x[2], Ys)
        evs[i][1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = nv.zkvc_kernel_launches() - launches0
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    return {"step_ms": step_ms, "tune_s": tune_s, "clocks": clk, "launches": launches, "batch": batch, "sets": sets,
            "Ys": Ys, "terms": batch.terms(), "info": batch.info()}


def plain_on_mix(nv, pks, instances, samples, rng):
    """The plain one-proof path on a request mix: zkvc_prove one instance at a time
    (inputs on the device, one warm call before each timed one), CUDA events."""
    import torch
    wss = {}
    out = []
    for _ in range(samples):
        k, Xd, Wd, rs = instances[rng.randrange(len(instances))]
        if k not in wss:
            wss[k] = torch.empty(nv.zkvc_prove_workspace_bytes(pks[k]), dtype=torch.uint8, device="cuda")
        nv.zkvc_prove(pks[k], Xd, Wd, rs, workspace=wss[k])  # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        nv.zkvc_prove(pks[k], Xd, Wd, rs, workspace=wss[k])
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    del wss
    torch.cuda.empty_cache()
    return {"proofs_per_s": 1e3 / statistics.mean(out), "p50_ms": statistics.median(out), "p99_ms": p99_of(out),
            "samples": len(out)}


def batched_section(nv, args, local):
    """The 64-proof batched workload inside the default bench line: proofs/s per graph
    replay, batch latency, and the plain one-proof path on the same 64 instances."""
    import random

    import torch

    from paper_2504_12217_gb300 import inputs
    shapes = inputs.batch_shapes()
    t0 = time.perf_counter()
    keys, _ = batched_setup(nv, inputs, shapes)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    steps = max(3, min(args.steps, 10))
    r = batched_core(nv, shapes, keys, steps, 2, local)
    step_ms = r["step_ms"]
    per = statistics.mean(step_ms)
    x = r["sets"][0]
    inst = [(i, x[0][i], x[1][i], x[2][i]) for i in range(len(shapes))]
    plain = plain_on_mix(nv, [keys[s] for s in shapes], inst, 64, random.Random(4))
    work = (r["terms"]["small"] + r["terms"]["main"]) * G1_MADD_PRODUCTS * MONT_IMAD + \
        r["terms"]["g2"] * G2_MADD_PRODUCTS * MONT_IMAD
    out = {"workload": "crpc_groth16_bn254_batched_64mix", "instances": len(shapes), "distinct_shapes": len(keys),
           "proofs_per_s": len(shapes) / (per / 1e3), "ms_per_batch_p50": statistics.median(step_ms),
           "ms_per_batch_p99": p99_of(step_ms), "steps": steps, "graph_kernels": r["info"]["graph_launches"],
           "gpu_launches": r["launches"], "tuning": r["batch"].get_tuning(), "tuning_source": "autotuned on the first call",
           "setup_s": setup_s, "autotune_and_capture_s": r["tune_s"], "whole_batch_imad_per_s": work / (per / 1e3),
           "plain_one_proof_path_same_64": plain, "clocks": r["clocks"],
           "l2": "flushed by a 256 MiB write between steps"}
    del r, keys
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    """64 seeded proofs of uneven [tokens, dim] x [dim, dim | 4 dim] shapes per step, one
    batched call (captured CUDA graph after autotuning).  One JSON line."""
    import torch

    from paper_2504_12217_gb300 import inputs
    from paper_2504_12217_gb300 import native as nv

    local = _env_int("LOCAL_RANK", 0)
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    shapes = inputs.batch_shapes(rank_seed(inputs.SEED_CFG[4], rank))
    if args.batch_count:  # a smaller case: the K smallest instances of the seeded mix
        shapes = sorted(shapes, key=lambda s: s[0] * s[1] + s[0] * s[2] + s[1] * s[2])[: args.batch_count]
    t0 = time.perf_counter()
    keys, vkeys = batched_setup(nv, inputs, shapes)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()
    r = batched_core(nv, shapes, keys, args.steps, args.warmup, local, tuning=args.tuning, eager=args.eager)
    if dist is not None:
        dist.barrier()
    batch, sets, Ys, step_ms = r["batch"], r["sets"], r["Ys"], r["step_ms"]
    total_s = reduce_max(sum(step_ms) / 1e3, dist, "cuda")
    count = len(shapes)
    value = replica_value(count * args.steps, world, total_s)
    terms = r["terms"]

    # end to end: pinned host matrices copied in, Y and proofs read back, every step
    Xh = [[x.cpu().pin_memory() for x in st[0]] for st in sets]
    Wh = [[w.cpu().pin_memory() for w in st[1]] for st in sets]
    Yh = [torch.empty(tuple(y.shape), dtype=torch.int32).pin_memory() for y in Ys]
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        x = sets[i % 2]
        for d, h in zip(x[0], Xh[i % 2]):
            d.copy_(h, non_blocking=True)
        for d, h in zip(x[1], Wh[i % 2]):
            d.copy_(h, non_blocking=True)
        batch.prove(x[0], x[1], x[2], Ys)
        for h, d in zip(Yh, Ys):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, dist, "cuda")
    h2d = sum(s[0] * s[1] + s[1] * s[2] for s in shapes)
    d2h = sum(256 + 4 * s[0] * s[2] for s in shapes)
    # parity spot check of the last step against the one-proof prover (not timed)
    x = sets[(args.steps - 1) % 2]
    proofs, _ = batch.prove(x[0], x[1], x[2], Ys)
    p0, _ = nv.zkvc_prove(keys[shapes[0]], x[0][0], x[1][0], x[2][0])
    # verification of the batch's proofs: batched on the GPU, and the host verifier on a few
    Yhost = [y.cpu().numpy() for y in Ys]
    Xhost = [t["X"] for t in x[3]]
    vlist = [vkeys[s] for s in shapes]
    nv.zkvc_verify_batch(vlist[:2], Xhost[:2], Yhost[:2], proofs[:2])  # warm (Frobenius table)
    t0 = time.perf_counter()
    vok = nv.zkvc_verify_batch(vlist, Xhost, Yhost, proofs)
    gpu_verify_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    host_ok = [nv.zkvc_verify(vlist[i], Xhost[i], Yhost[i], proofs[i]) for i in range(4)]
    host_verify_s = (time.perf_counter() - t0) / 4
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    imad = measure_imad_peak(nv, local)
    peak = imad["imad_per_s"] / 1e12
    work = (terms["small"] + terms["main"]) * G1_MADD_PRODUCTS * MONT_IMAD + terms["g2"] * G2_MADD_PRODUCTS * MONT_IMAD
    per_step = total_s / args.steps
    srt = sorted(step_ms)
    info = r["info"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 limbs (exact Fr/Fp arithmetic)", "data": "synthetic",
        "config": {"workload": "crpc_groth16_bn254_batched_64mix", "instances": count,
                   "distinct_shapes": len(keys), "shape_set": "a in {49,64,128,197}, n in {192,320,384,768}, b in {n,4n}",
                   "l2": "flushed by a 256 MiB write between steps", "parallelism": f"replicas x{world}",
                   "graph": not args.eager, "tuning": batch.get_tuning(),
                   "tuning_source": "imposed" if args.tuning else "autotuned on the first call"},
        "latency_ms": {"p50_batch": statistics.median(step_ms), "p99_batch": p99_of(step_ms), "min": srt[0],
                       "max": srt[-1]},
        "e2e": {"value": replica_value(count * e2e_steps, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "batch_roofline": {"bound": "alu", "scope": "whole batch (all kernels, overlapped)",
                           "achieved": work / per_step / 1e12, "peak": peak, "unit": "TIMAD/s",
                           "frac": work / per_step / 1e12 / peak, "bucket_terms": terms,
                           "peak_source": "measured on this GPU by zkvc_imad_rate (of measured)"},
        "gpu_launches": r["launches"], "gpu_launches_per_step": r["launches"] / args.steps,
        "graph_kernels": info["graph_launches"], "device_bytes": info["device_bytes"],
        "clocks": r["clocks"], "setup_s": setup_s, "autotune_and_capture_s": r["tune_s"],
        "spot_check_vs_one_proof_prover": proofs[0] == p0,
        "verify": {"gpu_batch_proofs_per_s": count / gpu_verify_s, "gpu_batch_s": gpu_verify_s,
                   "all_valid": all(vok), "host_ms_per_proof": host_verify_s * 1e3, "host_sample_valid": all(host_ok),
                   "note": "host wall clock; includes upload of keys, inputs and proofs"},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ served workload
def served_core(nv, pks, pool, rates, seconds_per_rate, max_requests, slots, budget, policy, local, rng):
    """Poisson arrivals (seeded) of requests drawn from `pool` through the library's proof
    server, one offered rate after the other.  Per rate: achieved proofs/s (requests over
    the time from the first arrival to the last result) and p50/p99 latency from submit
    to result (host wall clock, including the copies of X, W in and Y, the proof out)."""
    import threading
    srv = nv.Server(pks, slots=slots, mem_budget=budget, policy=policy)
    nv.zkvc_set_wait_timeout_ms(600000)
    for k in range(len(pks)):  # warm every key once (domain tables, side streams, caches)
        e = next(p for p in pool if p[0] == k)
        srv.wait(srv.submit(*e), k)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = nv.zkvc_kernel_launches()
    per_rate = []
    for rate in rates:
        n_req = max(8, min(max_requests, int(rate * seconds_per_rate)))
        arrivals, t = [], 0.0
        for _ in range(n_req):
            t += rng.expovariate(rate)
            arrivals.append(t)
        picks = [rng.randrange(len(pool)) for _ in range(n_req)]
        tickets = [None] * n_req
        results = [None] * n_req
        start = time.perf_counter()

        def collector():
            for i in range(n_req):
                while tickets[i] is None:
                    time.sleep(0.0002)
                k = pool[picks[i]][0]
                status, proof, _, times = srv.wait(tickets[i], k)
                results[i] = (status, times, time.perf_counter())

        th = threading.Thread(target=collector)
        th.start()
        for i in range(n_req):
            delay = start + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[i] = srv.submit(*pool[picks[i]])
        th.join()
        end = max(r[2] for r in results)
        lat = sorted(r[1]["total_ms"] for r in results)
        queue = sorted(r[1]["queue_ms"] for r in results)
        ok = sum(1 for r in results if r[0] == nv.ZKVC_OK)
        per_rate.append({"offered_rps": rate, "requests": n_req, "ok": ok,
                         "achieved_proofs_per_s": n_req / (end - start),
                         "p50_ms": statistics.median(lat), "p99_ms": p99_of(lat), "max_ms": lat[-1],
                         "queue_p50_ms": statistics.median(queue)})
    clk = clocks.stop()
    launches = nv.zkvc_kernel_launches() - launches0
    st = srv.stats()
    srv.close()
    return {"per_rate": per_rate, "clocks": clk, "launches": launches, "stats": st}


def served_pool(inputs, shapes, base_seed, rank=0):
    """Two pre-drawn instances per shape: (key index, X, W, rs)."""
    pool = []
    for k, s in enumerate(shapes):
        for v in range(2):
            seed = base_seed + 100 * k + v + 1000 * rank
            X, W = inputs.matrices(seed, *s)
            pool.append((k, X, W, inputs.to_bytes32(inputs.prover_values(seed))))
    return pool


def served_section(nv, args, local):
    """The served workload inside the default bench line: the 32 shapes' keys resident,
    Poisson arrivals at three offered rates (the highest above saturation) under two
    server policies -- chain (every request its own proof, overlapping on worker streams)
    and merge (queued requests proven together as merged batches) -- and the plain
    one-proof path on the same mix beside them."""
    import random

    import torch

    from paper_2504_12217_gb300 import inputs
    shapes = inputs.all_batch_shapes()
    t0 = time.perf_counter()
    pks = [nv.zkvc_setup(*s, inputs.to_bytes32(inputs.setup_values(shape_seed(inputs.SEED_CFG[5], s))))[0]
           for s in shapes]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    pool = served_pool(inputs, shapes, inputs.SEED_CFG[5])
    rng = random.Random(inputs.SEED_CFG[5])
    rates = args.served_rates
    runs = {}
    for name, policy, slots in (("chain", nv.ZKVC_SERVER_CHAIN, args.server_slots),
                                ("merge", nv.ZKVC_SERVER_MERGE, args.server_merge_slots)):
        r = served_core(nv, pks, pool, rates, args.served_seconds, args.served_max_requests, slots,
                        args.server_budget_gib << 30, policy, local, rng)
        best = max(r["per_rate"], key=lambda x: x["achieved_proofs_per_s"])
        runs[name] = {"slots": slots, "rates": r["per_rate"], "ceiling_proofs_per_s": best["achieved_proofs_per_s"],
                      "gpu_launches": r["launches"], "server_stats": r["stats"], "clocks": r["clocks"]}
    dev = [(k, torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(), rs) for k, X, W, rs in pool]
    plain = plain_on_mix(nv, pks, dev, 64, rng)
    del dev, pks
    torch.cuda.empty_cache()
    top = max(runs, key=lambda n: runs[n]["ceiling_proofs_per_s"])
    return {"workload": "crpc_groth16_bn254_served_poisson", "shapes": len(shapes),
            "mem_budget_bytes": args.server_budget_gib << 30, "policies": runs,
            "ceiling_proofs_per_s": runs[top]["ceiling_proofs_per_s"], "ceiling_policy": top,
            "plain_one_proof_path_same_mix": plain, "setup_s": setup_s,
            "latency": "host wall clock from submit to result (includes H2D of X, W and D2H of Y, proof)"}


def run_served(args):
    """Poisson arrivals (seeded) of proof requests over the 32 [tokens, dim] x [dim, dim |
    4 dim] shapes, all keys resident; the library's proof server admits requests by
    memory footprint and overlaps them.  Per offered rate: achieved proofs/s and p50/p99
    latency from submission to result.  The plain path (one proof at a time through
    zkvc_prove, inputs already on the device) on the same request mix is reported beside
    it.  One JSON line."""
    import random

    import torch

    from paper_2504_12217_gb300 import inputs
    from paper_2504_12217_gb300 import native as nv

    local = _env_int("LOCAL_RANK", 0)
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    torch.cuda.set_device(local)
    shapes = inputs.all_batch_shapes()
    t0 = time.perf_counter()
    pks = [nv.zkvc_setup(*s, inputs.to_bytes32(inputs.setup_values(shape_seed(inputs.SEED_CFG[5], s))))[0]
           for s in shapes]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    pool = served_pool(inputs, shapes, inputs.SEED_CFG[5], rank)
    rng = random.Random(inputs.SEED_CFG[5] + rank)
    policy = {"adaptive": nv.ZKVC_SERVER_ADAPTIVE, "fold": nv.ZKVC_SERVER_FOLD, "chain": nv.ZKVC_SERVER_CHAIN,
              "merge": nv.ZKVC_SERVER_MERGE}[args.server_policy]
    budget = args.server_budget_gib << 30
    r = served_core(nv, pks, pool, args.rates, args.seconds_per_rate, args.max_requests, args.server_slots, budget,
                    policy, local, rng)
    dev = [(k, torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(), rs) for k, X, W, rs in pool]
    plain = plain_on_mix(nv, pks, dev, 64, rng)
    if rank != 0:
        return 0
    per_rate = r["per_rate"]
    best = max(per_rate, key=lambda x: x["achieved_proofs_per_s"])
    line = {
        "metric": METRIC, "value": best["achieved_proofs_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": sum(x["requests"] for x in per_rate), "warmup": len(shapes), "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 limbs (exact Fr/Fp arithmetic)", "data": "synthetic",
        "config": {"workload": "crpc_groth16_bn254_served_poisson", "shapes": len(shapes),
                   "rates_rps": args.rates, "slots": args.server_slots, "mem_budget_bytes": budget,
                   "policy": {"adaptive": "adaptive (fold when idle, chain when shared)", "fold": "fold",
                              "chain": "chain", "merge": "merge (queued requests in merged batches)"}[
                                  args.server_policy],
                   "latency": "host wall clock from submit to result (includes H2D of X, W and D2H of Y, proof)"},
        "served": per_rate,
        "plain_one_proof_path": plain,
        "server_stats": r["stats"], "gpu_launches": r["launches"], "clocks": r["clocks"], "setup_s": setup_s,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ablation (Table II)
def run_ablation(args):
    """The paper's ablation (Sec. V, Table II) on the GPU: one [49,320] x [320,512] proof
    per circuit encoding (vanilla, PSQ only, CRPC only, CRPC + PSQ) through the generic
    sparse-R1CS prover, the specialised CRPC + PSQ prover in both modes, and the
    private-input variant.  Device-timed (CUDA events), L2 flushed between steps.  One
    JSON line; value = proofs/s of the specialised CRPC + PSQ prover (fold mode)."""
    import torch

    from paper_2504_12217_gb300 import inputs
    from paper_2504_12217_gb300 import native as nv

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    a, n, b = SHAPE
    inst = inputs.instance(inputs.SEED_CFG[2], SHAPE)
    Xd = torch.from_numpy(inst["X"]).cuda()
    Wd = torch.from_numpy(inst["W"]).cuda()
    rs = inputs.to_bytes32(inst["rs"])
    toxic = inputs.to_bytes32(inst["toxic"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        out = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    rows = []
    variants = [("vanilla", "xy"), ("psq", "xy"), ("crpc", "xy"), ("crpc_psq", "xy"), ("crpc_psq", "none"),
                ("vanilla", "none")]
    for circuit, pub in variants:
        t0 = time.perf_counter()
        pk, vk = nv.zkvc_setup_circuit(a, n, b, circuit, pub, toxic)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        info = nv.zkvc_pk_circuit(pk)
        ws = torch.empty(nv.zkvc_prove_workspace_bytes(pk), dtype=torch.uint8, device="cuda")
        Y = torch.empty((a, b), dtype=torch.int32, device="cuda")
        steps = args.steps if info["rows"] < (1 << 20) else max(3, args.steps // 5)
        ms = timed(lambda: nv.zkvc_prove(pk, Xd, Wd, rs, Y=Y, workspace=ws), steps)
        proof, _ = nv.zkvc_prove(pk, Xd, Wd, rs, Y=Y, workspace=ws)
        t0 = time.perf_counter()
        ok = nv.zkvc_verify(vk, inst["X"] if pub == "xy" else None, Y.cpu().numpy() if pub == "xy" else None, proof)
        verify_ms = (time.perf_counter() - t0) * 1e3
        rows.append({"circuit": circuit, "public_io": pub, "engine": "generic", "r1cs_rows": info["rows"],
                     "variables": info["vars"], "log_domain": pk.log_domain, "prove_ms": ms, "setup_s": setup_s,
                     "verify_ms_host": verify_ms, "verified": ok})
        del pk, vk, ws
        torch.cuda.empty_cache()
    pk, vk = nv.zkvc_setup(a, n, b, toxic)
    for mode, name in ((nv.ZKVC_PROVE_FOLD, "fold"), (nv.ZKVC_PROVE_CHAIN, "chain")):
        ws = torch.empty(nv.zkvc_prove_workspace_bytes_mode(pk, mode), dtype=torch.uint8, device="cuda")
        Y = torch.empty((a, b), dtype=torch.int32, device="cuda")
        ms = timed(lambda: nv.zkvc_prove_mode(pk, mode, Xd, Wd, rs, Y=Y, workspace=ws), args.steps)
        rows.append({"circuit": "crpc_psq", "public_io": "xy", "engine": f"specialised ({name})",
                     "r1cs_rows": n + a * n + a * b + 1, "log_domain": pk.log_domain, "prove_ms": ms})
    base = next(r for r in rows if r["engine"] == "specialised (fold)")["prove_ms"]
    line = {
        "metric": METRIC, "value": 1e3 / base, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": base, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 limbs (exact Fr/Fp arithmetic)", "data": "synthetic",
        "config": {"workload": "crpc_groth16_bn254_ablation_49x320x512", "a": a, "n": n, "b": b,
                   "l2": "flushed by a 256 MiB write between steps"},
        "ablation": rows,
        "paper_table2_cpu_s": {"vanilla": 9.12, "psq": 8.69, "crpc": 1.01, "crpc_psq": 0.73,
                               "note": "16-core CPU, a patch-embedding matmul of unstated size; context only"},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plain: skip zkvc_pk_autotune at setup (default MSM chunk rule)")
    ap.add_argument("--sweep", action="store_true", help="kernel sweep (NTT and MSM sizes) instead of proofs")
    ap.add_argument("--sweep-ntt", type=int, nargs="*", default=[16, 18, 20, 22, 24])
    ap.add_argument("--sweep-g1", type=int, nargs="*", default=[16, 18, 20, 22, 24])
    ap.add_argument("--sweep-g2", type=int, nargs="*", default=[16, 18, 20])
    ap.add_argument("--workload", choices=["plain", "batched", "served", "ablation"], default="plain",
                    help="plain: one [49,320]x[320,512] proof per step; batched: 64 mixed shapes per step; "
                         "served: Poisson arrivals over 32 shapes through the proof server")
    ap.add_argument("--rates", type=float, nargs="*", default=[1, 2, 5, 10, 20, 50, 100, 200])
    ap.add_argument("--seconds-per-rate", type=float, default=6.0)
    ap.add_argument("--max-requests", type=int, default=1200)
    ap.add_argument("--server-slots", type=int, default=8)
    ap.add_argument("--server-budget-gib", type=int, default=48)
    ap.add_argument("--server-policy", choices=["adaptive", "fold", "chain", "merge"], default="chain",
                    help="served: prover mode per request, or merged batches of queued requests")
    ap.add_argument("--server-merge-slots", type=int, default=3,
                    help="plain: workers of the merge-policy server in the served section")
    ap.add_argument("--batch-count", type=int, default=0, help="batched: only the K smallest instances")
    ap.add_argument("--no-batched", action="store_true", help="plain: leave the batched section out of the line")
    ap.add_argument("--no-served", action="store_true", help="plain: leave the served section out of the line")
    ap.add_argument("--no-msm-sweep", action="store_true", help="plain: leave the MSM sweep points out of the line")
    ap.add_argument("--served-rates", type=float, nargs="*", default=[50, 200, 1000],
                    help="plain: offered rates of the served section (the last above saturation)")
    ap.add_argument("--served-seconds", type=float, default=3.0, help="plain: seconds of arrivals per served rate")
    ap.add_argument("--served-max-requests", type=int, default=600, help="plain: request cap per served rate")
    ap.add_argument("--key-tuning", type=int, nargs=10, default=None,
                    help="plain: impose the key's launch shape (zkvc_pk_set_tuning), skip the autotuner")
    ap.add_argument("--tuning", type=int, nargs=7, default=None, help="batched: impose a tuning, skip the autotuner")
    ap.add_argument("--eager", action="store_true", help="batched: launch eagerly instead of replaying a graph")
    args = ap.parse_args()
    if args.sweep:
        return run_sweep(args)
    if args.workload == "batched" and args.impl == "ours":
        return run_batched(args)
    if args.workload == "served" and args.impl == "ours":
        return run_served(args)
    if args.workload == "ablation" and args.impl == "ours":
        return run_ablation(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
