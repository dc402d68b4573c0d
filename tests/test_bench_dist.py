"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their step
times (max) and processed units (sum) into the whole-job rate."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier()
        units = 1000.0 * (rank + 1)
        ms = 10.0 + 5.0 * rank
        rate, total, ms_max = bench.whole_job_rate(units, ms)
        mx = bench.dist_reduce([rank, -rank], "max")
        sm = bench.dist_reduce([rank, 1.0], "sum")
        out.put((rank, rate, total, ms_max, mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_whole_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, total, ms_max, mx, sm in res:
        assert total == 3000.0
        assert ms_max == 15.0
        assert rate == pytest.approx(3000.0 / 0.015)
        assert mx == [1.0, 0.0]
        assert sm == [1.0, 2.0]


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_reduce([3, 4.5], "max") == [3.0, 4.5]
    rate, units, ms = bench.whole_job_rate(500.0, 250.0)
    assert (rate, units, ms) == (2000.0, 500.0, 250.0)
