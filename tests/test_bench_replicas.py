"""The multi-GPU bench path (independent replicas) on CPU: two gloo ranks agree on the slowest
rank's time, and the whole-job value counts every rank's units over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
        dist.barrier()
        t_max = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        results[rank] = (t_max, bench.whole_job_value(1000.0, 4, world, t_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        results = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, results)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        got = dict(results)
    assert got[0][0] == got[1][0] == 150.0
    # 2 ranks x 4 steps x 1000 units in 0.15 s
    assert abs(got[0][1] - 2 * 4 * 1000.0 / 0.15) < 1e-6


def test_single_rank_is_its_own_max():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(42.0, 1, None) == 42.0
    assert bench.whole_job_value(10.0, 2, 1, 1000.0) == 20.0
