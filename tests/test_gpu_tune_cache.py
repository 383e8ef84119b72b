"""The one-proof autotuner's cache on the GPU: a second key of the same shape takes the
first key's tuned launch shape without timing (and proves the oracle's bytes with it);
ZKVC_TUNE_FRESH tunes again; a saved cache, loaded into a cleared one, serves the key."""
import time

import pytest

from oracle import crpc, groth16 as og
from paper_2504_12217_gb300 import inputs
from tests import _util

pytestmark = pytest.mark.gpu


def test_tuning_cache_serves_same_shape(tmp_path):
    import torch
    assert torch.cuda.is_available()
    nv = _util.native()
    a, n, b = 5, 7, 3
    nv.zkvc_tune_cache_clear()
    insts = [inputs.instance(9100 + i, (a, n, b)) for i in range(2)]
    keys = [nv.zkvc_setup(a, n, b, inputs.to_bytes32(t["toxic"]))[0] for t in insts]
    dev = [(torch.from_numpy(t["X"]).cuda(), torch.from_numpy(t["W"]).cuda(), inputs.to_bytes32(t["rs"])) for t in insts]
    t0 = time.perf_counter()
    first = nv.zkvc_pk_autotune(keys[0], *dev[0], mode=nv.ZKVC_PROVE_AUTO)
    tuned_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    second = nv.zkvc_pk_autotune(keys[1], *dev[1], mode=nv.ZKVC_PROVE_AUTO)
    cached_s = time.perf_counter() - t0
    assert second == first and nv.zkvc_pk_get_tuning(keys[1]) == first
    assert cached_s < tuned_s / 5
    proof, _ = nv.zkvc_prove(keys[1], *dev[1])
    X, W = insts[1]["X"].astype(int).tolist(), insts[1]["W"].astype(int).tolist()
    cf, _ = og.closed_form_proof(crpc.Shape(a, n, b), insts[1]["toxic"], X, W, *insts[1]["rs"])
    assert proof == og.proof_bytes(cf)
    path = tmp_path / "tune.txt"
    nv.zkvc_tune_cache_save(path)
    nv.zkvc_tune_cache_clear()
    nv.zkvc_tune_cache_load(path)
    t0 = time.perf_counter()
    assert nv.zkvc_pk_autotune(keys[0], *dev[0], mode=nv.ZKVC_PROVE_AUTO) == first
    assert time.perf_counter() - t0 < tuned_s / 5
    t0 = time.perf_counter()
    nv.zkvc_pk_autotune(keys[0], *dev[0], mode=nv.ZKVC_PROVE_AUTO, fresh=True)
    assert time.perf_counter() - t0 > cached_s
    nv.zkvc_tune_cache_clear()
