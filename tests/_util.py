"""Test helpers: byte conversions between Python integers and uint8 tensors, and the
loader of the CUDA library (built in-tree on first use)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zkvc.h")


def native():
    from paper_2504_12217_gb300 import build, native as nv
    if not os.path.exists(nv.LIB_PATH):
        build.build()
    nv.lib()
    return nv


def declared_functions():
    """Function names declared in include/zkvc.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zkvc_\w+)\s*\(", text)))


def ints_to_u8(values, width=32):
    buf = b"".join(int(v).to_bytes(width, "little") for v in values)
    return np.frombuffer(buf, dtype=np.uint8).reshape(len(values), width).copy()


def u8_to_ints(arr, width=32):
    raw = bytes(np.ascontiguousarray(arr).reshape(-1))
    return [int.from_bytes(raw[i:i + width], "little") for i in range(0, len(raw), width)]


def to_cuda(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def g1_rows(points):
    from oracle import bn254 as bn
    return np.frombuffer(b"".join(bn.g1_bytes(p) for p in points), dtype=np.uint8).reshape(len(points), 64).copy()


def g2_rows(points):
    from oracle import bn254 as bn
    return np.frombuffer(b"".join(bn.g2_bytes(p) for p in points), dtype=np.uint8).reshape(len(points), 128).copy()
