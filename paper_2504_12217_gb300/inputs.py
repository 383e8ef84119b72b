"""Seeded synthetic inputs for the CRPC-matmul Groth16 workloads.

This module only draws random numbers; it holds none of the proof system's arithmetic.
Both the CUDA path and the oracle receive what it draws as plain inputs:

* the int8 matrices X (a x n) and W (n x b), uniform over [-128, 127];
* the Groth16 toxic waste (tau, alpha, beta, gamma, delta) and the CRPC point z, passed
  to setup as six 32-byte little-endian values;
* the prover randomness (r, s), passed to prove as two 32-byte values.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used in counter form: output k (k = 1, 2, ...) of a stream
is mix(state0 + k * 0x9E3779B97F4A7C15 mod 2^64).  A stream is named by (seed, tag) with
state0 = seed XOR (tag * 0x9E3779B97F4A7C15 mod 2^64).  Tags: 1 = matrix data (X
row-major then W row-major, one word per entry, low byte as two's-complement int8),
2 = setup values (tau, alpha, beta, gamma, delta, z), 3 = prover values (r, s),
4 = shape draws of the batched workload.

A field-sized draw takes four consecutive words little-endian and keeps the low 253 bits,
so it is below the BN254 group order (> 2^253) without rejection.
"""
import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
TAG_DATA, TAG_SETUP, TAG_PROVER, TAG_SHAPES = 1, 2, 3, 4

# workload seeds: configuration k uses 0x5A4B5643_0000000k
SEED_CFG = {k: (0x5A4B5643 << 32) | k for k in range(1, 6)}

# matmul shapes (a, n, b) = (tokens, inner, out)
SHAPE_CFG1 = (4, 16, 8)
SHAPE_CFG2 = (49, 320, 512)
BATCH_TOKENS = (49, 64, 128, 197)
BATCH_DIMS = (192, 320, 384, 768)
BATCH_COUNT = 64


def _mix(z):
    """SplitMix64 output function on a uint64 numpy array (wrapping arithmetic)."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def words(seed, tag, count, start=0):
    """Words start+1 .. start+count of stream (seed, tag) as uint64."""
    state0 = np.uint64((seed ^ ((tag * GOLDEN) & MASK64)) & MASK64)
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(state0 + k * np.uint64(GOLDEN))


def matrices(seed, a, n, b):
    """X (a x n) and W (n x b) as int8 numpy arrays, row-major, from tag 1."""
    w = words(seed, TAG_DATA, a * n + n * b)
    lo = (w & np.uint64(0xFF)).astype(np.uint8).view(np.int8)
    X = lo[: a * n].reshape(a, n).copy()
    W = lo[a * n:].reshape(n, b).copy()
    return X, W


def field_draws(seed, tag, count):
    """count values of 253 bits each (four words little-endian, top 3 bits cleared)."""
    w = words(seed, tag, 4 * count)
    out = []
    for i in range(count):
        v = 0
        for j in range(4):
            v |= int(w[4 * i + j]) << (64 * j)
        out.append(v & ((1 << 253) - 1))
    return out


def setup_values(seed):
    """(tau, alpha, beta, gamma, delta, z) as Python ints."""
    return field_draws(seed, TAG_SETUP, 6)


def prover_values(seed):
    """(r, s) as Python ints."""
    return field_draws(seed, TAG_PROVER, 2)


def to_bytes32(values):
    """Concatenated 32-byte little-endian encodings (the C-ABI's input format)."""
    return b"".join(int(v).to_bytes(32, "little") for v in values)


def batch_shapes(seed=SEED_CFG[4], count=BATCH_COUNT):
    """Shapes (a, n, b) of the batched workload: a from the token set, n from the
    dimension set, b in {n, 4n}, one draw of three words per instance (tag 4)."""
    w = words(seed, TAG_SHAPES, 3 * count)
    shapes = []
    for i in range(count):
        a = BATCH_TOKENS[int(w[3 * i]) % len(BATCH_TOKENS)]
        n = BATCH_DIMS[int(w[3 * i + 1]) % len(BATCH_DIMS)]
        b = n * (1 if int(w[3 * i + 2]) % 2 == 0 else 4)
        shapes.append((a, n, b))
    return shapes


def all_batch_shapes():
    """The 32 distinct shapes of the batched / served workloads."""
    return [(a, n, n * m) for a in BATCH_TOKENS for n in BATCH_DIMS for m in (1, 4)]


def instance(seed, shape):
    """Everything one proof needs: X, W, toxic waste and (r, s)."""
    a, n, b = shape
    X, W = matrices(seed, a, n, b)
    return {"shape": shape, "X": X, "W": W, "toxic": setup_values(seed), "rs": prover_values(seed)}
