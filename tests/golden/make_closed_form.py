"""Writes the expected full-size Groth16 proofs that the GPU parity tests compare with.

Every value here comes from ``oracle.groth16.closed_form_proof`` (Sec. II Prove, with the
toxic waste in the exponent: each MSM of the proof collapses to one scalar multiple of
the generator) on inputs drawn by ``paper_2504_12217_gb300.inputs`` (seeded SplitMix64,
no arithmetic of the method).  Y is passed to the oracle as numpy's exact int64 product
X W, a library primitive standing in for the oracle's pure-Python triple loop, which
would take minutes at the largest shapes.

Two files:

* ``closed_form_49x320x512.txt``: the [49,320]x[320,512] instance of the one-proof
  benchmark (seed 0x5A4B5643_00000002, its setup values and matrices) proven with the
  prover values of seeds seed * 1000 + i, i = 0 .. 7, the (r, s) sequence the benchmark
  draws for its steps.  Line: ``i r s proof`` (hex).
* ``closed_form_batch64.txt``: the 64 instances of the batched workload (shapes drawn
  with seed 0x5A4B5643_00000004, one key per distinct shape from setup seed
  base ^ (a << 40) ^ (n << 20) ^ b, instance i from seed base + 1000 + i).  Line:
  ``i a n b proof`` (hex).

Run from the repository root: ``python tests/golden/make_closed_form.py`` (all host
cores, a few minutes).
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CFG2_STEPS = 8


def batch_shape_seed(base, shape):
    a, n, b = shape
    return base ^ (a << 40) ^ (n << 20) ^ b


def _proof(job):
    import numpy as np

    from oracle import crpc
    from oracle import groth16 as og
    from paper_2504_12217_gb300 import inputs

    kind, i, shape, toxic_seed, data_seed, rs_seed = job
    X, W = inputs.matrices(data_seed, *shape)
    toxic = inputs.setup_values(toxic_seed)
    r, s = inputs.prover_values(rs_seed)
    Y = (X.astype(np.int64) @ W.astype(np.int64)).tolist()
    cf, _ = og.closed_form_proof(crpc.Shape(*shape), toxic, X.astype(int).tolist(), W.astype(int).tolist(), r, s,
                                 Y=Y)
    return kind, i, shape, r, s, og.proof_bytes(cf).hex()


def jobs():
    from paper_2504_12217_gb300 import inputs

    out = []
    seed2 = inputs.SEED_CFG[2]
    for i in range(CFG2_STEPS):
        out.append(("cfg2", i, inputs.SHAPE_CFG2, seed2, seed2, seed2 * 1000 + i))
    base = inputs.SEED_CFG[4]
    for i, shape in enumerate(inputs.batch_shapes(base)):
        seed = base + 1000 + i
        out.append(("batch", i, shape, batch_shape_seed(base, shape), seed, seed))
    # largest shapes first so that the pool's tail is short
    out.sort(key=lambda j: -(j[2][0] * j[2][1] + j[2][0] * j[2][2] + j[2][1] * j[2][2]))
    return out


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count() or 4) as pool:
        res = pool.map(_proof, jobs(), chunksize=1)
    cfg2 = sorted(r for r in res if r[0] == "cfg2")
    batch = sorted(r for r in res if r[0] == "batch")
    with open(os.path.join(HERE, "closed_form_49x320x512.txt"), "w") as fh:
        fh.write("# Groth16 proofs (Sec. II) of the [49,320]x[320,512] CRPC + PSQ instance, seed 0x5A4B5643_00000002,\n"
                 "# prover values of seeds seed * 1000 + i; oracle closed form; written by make_closed_form.py\n"
                 "# i r s proof(A 64 B | B 128 B | C 64 B)\n")
        for _, i, _, r, s, p in cfg2:
            fh.write(f"{i} {r:064x} {s:064x} {p}\n")
    with open(os.path.join(HERE, "closed_form_batch64.txt"), "w") as fh:
        fh.write("# Groth16 proofs (Sec. II) of the 64 batched CRPC + PSQ instances, seed 0x5A4B5643_00000004;\n"
                 "# oracle closed form; written by make_closed_form.py\n"
                 "# i a n b proof(A 64 B | B 128 B | C 64 B)\n")
        for _, i, (a, n, b), _, _, p in batch:
            fh.write(f"{i} {a} {n} {b} {p}\n")


if __name__ == "__main__":
    main()
