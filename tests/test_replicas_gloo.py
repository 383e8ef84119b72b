"""The multi-GPU form is replicas only (proofs are independent): each rank proves its own
seeded instances and the job's throughput is all ranks' proofs over the slowest rank's
time.  This checks that host logic with two gloo ranks on the CPU: the max-over-ranks
reduction, the whole-job value, and that ranks draw disjoint inputs."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from paper_2504_12217_gb300 import inputs

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 1.0 + 0.5 * rank  # rank 1 is the slower one
        tmax = bench.reduce_max(local_s, dist, "cpu")
        seed = bench.rank_seed(inputs.SEED_CFG[2], rank)
        X, _ = inputs.matrices(seed, 4, 16, 8)
        shapes = inputs.batch_shapes(bench.rank_seed(inputs.SEED_CFG[4], rank), 8)
        objs = [None] * world
        dist.all_gather_object(objs, (seed, X.tobytes(), shapes))
        out[rank] = (tmax, bench.replica_value(10, world, tmax), objs)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for rank in range(2):
        tmax, value, objs = res[rank]
        assert tmax == pytest.approx(1.5)
        assert value == pytest.approx(2 * 10 / 1.5)
        (s0, x0, sh0), (s1, x1, sh1) = objs
        assert s0 != s1 and x0 != x1 and sh0 != sh1


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(2.25, None, "cpu") == 2.25
    assert bench.replica_value(64, 1, 0.2) == pytest.approx(320.0)
