"""The primitives of a state held over several GPUs, through the C ABI, and
the sharded state itself with the library as each rank's engine.

sv_select_histogram must give, for every prefix of the canonical composite
Z = (~prob bits, natural key), the exact counts and fixed-point masses of the
next digit (checked against the oracle's probabilities); sv_cut must keep the
terms up to a composite with the global masses' renormalisation (checked
against the oracle's truncation of the same state).  Then two ranks, each a
process with its own handle on cuda:0 (collectives on the host through gloo,
no kernel waits on another process), run a circuit whose gates touch the
partition qubit; their union must equal the oracle run alone, bit for bit.
"""
import os
import socket
import struct
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2607_07816_b300 import circuits as C

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import sv as _sv
    _sv.load_library()
    return _sv


def _zs(oracle_mod, o):
    k, a, p = o.export()
    z = [(((~struct.unpack("<Q", struct.pack("<d", float(x)))[0]) & (2 ** 64 - 1)) << 64) | int(kk)
         for x, kk in zip(p, k)]
    return k, a, p, z


@pytest.mark.parametrize("prec", [0, 1])
def test_select_histogram_levels_match_the_oracle(sv, oracle_mod, prec):
    rng = np.random.default_rng(7700 + prec)
    keys, amps = C.random_state(30, 50_000, rng, ties=True)
    g = sv.SparseState(30, prec=prec)
    o = oracle_mod.Oracle(30, prec=prec)
    g.load(keys, amps)
    o.load(keys, amps)
    _, _, p, zs = _zs(oracle_mod, o)
    fxs = [oracle_mod.fx(float(x)) for x in p]
    prefix, bits = 0, 0
    while bits < 128:
        counts, masses = g.select_histogram(prefix, bits)
        D = min(11, 128 - bits)
        shift = 128 - bits - D
        wc, wm = [0] * 2048, [0] * 2048
        for z, f in zip(zs, fxs):
            if bits and (z >> (128 - bits)) != (prefix >> (128 - bits)):
                continue
            d = (z >> shift) & ((1 << D) - 1)
            wc[d] += 1
            wm[d] += f
        assert counts.tolist() == wc, bits
        assert masses == wm, bits
        # descend into the most populated bin
        d = int(np.argmax(counts))
        if counts[d] <= 1:
            break
        prefix |= d << shift
        bits += D
    # exact probability ties: with the whole probability fixed (64 bits) the
    # next digits are key bits, and the bin counts add up to the multiplicity
    vals, mult = np.unique(np.asarray(p, dtype=np.float64), return_counts=True)
    tied = float(vals[int(np.argmax(mult))])
    assert mult.max() >= 2
    pb = struct.unpack("<Q", struct.pack("<d", tied))[0]
    for bits in (64, 75):
        prefix = ((~pb) & (2 ** 64 - 1)) << 64
        if bits == 75:
            key0 = min(int(z) & (2 ** 64 - 1) for z in zs if z >> 64 == prefix >> 64)
            prefix |= (key0 >> 53) << 53
        counts, masses = g.select_histogram(prefix, bits)
        want = sum(1 for z in zs if (z >> (128 - bits)) == (prefix >> (128 - bits)))
        assert int(counts.sum()) == want and want >= 1, bits
        assert sum(masses) == want * oracle_mod.fx(tied), bits


@pytest.mark.parametrize("prec", [0, 1])
def test_cut_matches_the_oracle_truncation(sv, oracle_mod, prec):
    rng = np.random.default_rng(7800 + prec)
    keys, amps = C.random_state(40, 30_000, rng, ties=True)
    for K in (1, 777, 12_345, 29_999):
        g = sv.SparseState(40, prec=prec)
        g.load(keys, amps)
        o = oracle_mod.Oracle(40, K, 1.0, prec=prec)
        o.load(keys, amps)
        _, _, _, zs = _zs(oracle_mod, o)
        z_cut = sorted(zs)[K - 1]
        S_N = o.total_mass_fx()
        o.truncate()
        S_c = o.last_cut()["Sc"]
        kept = g.cut(z_cut, S_c, S_N)
        assert kept == K
        gk, ga = g.export()
        ok, oa, _ = o.export()
        assert np.array_equal(gk, ok) and np.array_equal(ga, oa)
        assert g.retained_mass() == o.retained_mass()
        assert g.peak() == o.peak()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, prec, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2607_07816_b300 import sv
    from paper_2607_07816_b300.shard import ShardedState
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        c = C.random_mix_circuit(24, 40, seed=91 + prec, sigma=0.05, K=3000, p=0.999)
        sh = ShardedState(c.n, c.K, c.p, lambda n: sv.SparseState(n, 1 << 62, 1.0, prec=prec))
        ref = oracle.Oracle(c.n, c.K, c.p, prec=prec)
        bad = []
        swaps = 0
        for t, (q, u) in enumerate(c.gates):
            before = list(sh.glob)
            sh.apply_gate(q, u)
            swaps += sh.glob != before
            ref.apply_gate(q, u)
            if sh.truncate() != ref.truncate():
                bad.append((t, "truncate"))
            k, a = sh.export()
            rk, ra, _ = ref.export()
            if dict(zip(k.tolist(), a.tolist())) != dict(zip(rk.tolist(), ra.tolist())):
                bad.append((t, "state"))
            if sh.peak() != ref.peak():
                bad.append((t, "peak"))
            if bad:
                break
        out.put((rank, bad, swaps, sh.retained_mass() == ref.retained_mass()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("prec", [0, 1])
def test_two_ranks_on_one_gpu_equal_the_oracle(sv, prec):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, prec, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=900) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, bad, swaps, same_F in res:
        assert not bad, (rank, bad[:3])
        assert swaps > 0
        assert same_F
