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


def test_amp_error_and_peaked_check():
    """The complex64-vs-complex128 comparison of the serving legs: amplitude
    error on the common keys, the keys held by one side only, and the peak
    counts restricted to the peaked requests."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    ka = np.array([1, 5, 9], dtype=np.uint64)
    aa = np.array([0.6, 0.8j, 1e-3], dtype=np.complex64)
    kb = np.array([9, 1, 7, 5], dtype=np.uint64)
    ab = np.array([1e-3, 0.6 + 1e-6, 0.01, 0.8j], dtype=np.complex128)
    err, nd, mass = bench.amp_error(ka, aa, kb, ab)
    assert err == pytest.approx(1e-6, rel=0.2, abs=3e-8)  # float32 rounding of 0.6 is ~2e-8
    assert nd == 1 and mass == pytest.approx(1e-4)

    class R:
        def __init__(self, key, keys=None, amps=None):
            self.peak_key, self.keys, self.amps = key, keys, amps

    serial = [{"key": 1, "gap": 0.5, "F": 0.9, "keys": kb, "amps": ab},  # peaked
              {"key": 2, "gap": 1e-5, "F": 0.9},                          # no clear top
              {"key": 3, "gap": 0.5, "F": 1e-9}]                          # mass too small
    batched = [R(1), R(4), R(3)]
    chk = [R(1, ka, aa), None, None]
    out = bench.peaked_check(batched, serial, [None] * 3, chk)
    assert out["peaked_requests"] == 1 and out["identical_peaks_on_peaked"] == "1/1"
    assert out["identical_peaks_all"] == "2/3"
    chk_out = out["amp_check_on_peaked"]
    assert chk_out["different_kept_set"]["within_tol"] == "1/1"  # key 7 is held by one side only
    assert chk_out["same_kept_set"] == {"requests": 0}
