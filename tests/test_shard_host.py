"""One state held over several ranks (paper_2607_07816_b300.shard), on CPU.

Two and four gloo ranks each hold a partition of the terms; the per-rank
engine is the CPU oracle wrapped with the two primitives the sharded
truncation needs (the select histogram of the composite and the cut at a
given composite, written here from their definitions).  After every gate
and truncation the union of the ranks' terms must equal the oracle run on
the whole state alone, bit for bit: the partition-bit exchanges, the radix
select summed over the ranks and the global renormalisation reproduce the
single-state rule of Sec. III exactly.
"""
import math
import os
import socket
import struct
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TWO120 = 1 << 120


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleEngine:
    """The oracle with the shard primitives: Z = (~prob bits, key) digits and
    the cut with the global masses (Sec. III, R6-R8)."""

    def __init__(self, oracle_mod, n, prec=0):
        self.om = oracle_mod
        self.o = oracle_mod.Oracle(n, 1 << 62, 1.0, prec=prec)
        self.prec = prec
        self.F = 1.0

    def apply_gate(self, q, u):
        self.o.apply_gate(q, u)

    def num_terms(self):
        return self.o.num_terms()

    def export(self):
        k, a, _ = self.o.export()
        return k.copy(), a.copy()

    def load(self, keys, amps):
        self.o.load(keys, amps)

    def _z(self):
        k, a, p = self.o.export()
        bits = [struct.unpack("<Q", struct.pack("<d", float(x)))[0] for x in p]
        return k, a, [((~b & (2 ** 64 - 1)) << 64) | int(kk) for b, kk in zip(bits, k)], p

    def select_histogram(self, prefix, bits):
        D = min(11, 128 - bits)
        shift = 128 - bits - D
        counts = [0] * 2048
        masses = [0] * 2048
        _, _, zs, p = self._z()
        for z, pr in zip(zs, p):
            if bits and (z >> (128 - bits)) != (prefix >> (128 - bits)):
                continue
            d = (z >> shift) & ((1 << D) - 1)
            counts[d] += 1
            masses[d] += self.om.fx(float(pr))
        return np.array(counts, dtype=np.uint32), masses

    def cut(self, zc, S_c, S_N):
        k, a, zs, _ = self._z()
        keep = [i for i, z in enumerate(zs) if z <= zc]
        s = 1.0 / math.sqrt(self.om.fx_to_double(S_c))
        out = []
        for i in keep:
            x = a[i]
            if self.prec == 0:
                out.append(complex(x.real * s, x.imag * s))
            else:
                out.append(complex(float(np.float32(x.real * s)), float(np.float32(x.imag * s))))
        self.o.load(k[keep], np.array(out, dtype=np.complex128))
        self.F *= self.om.fx_to_double(S_c) / self.om.fx_to_double(S_N)
        return len(keep)

    def peak(self):
        return self.o.peak()

    def retained_mass(self):
        return self.F


def _rank(rank, world, port, case, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300.shard import ShardedState
    oracle.build()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        c = _circuit(C, case)
        sh = ShardedState(c.n, c.K, c.p, lambda n: OracleEngine(oracle, n, case["prec"]))
        ref = oracle.Oracle(c.n, c.K, c.p, prec=case["prec"])
        bad = []
        most = 0
        for t, (q, u) in enumerate(c.gates):
            sh.apply_gate(q, u)
            ref.apply_gate(q, u)
            got = sh.truncate()
            want = ref.truncate()
            most = max(most, sh.eng.num_terms())
            if got != want:
                bad.append((t, "truncate", got, want))
            k, a = sh.export()
            rk, ra, _ = ref.export()
            if dict(zip(k.tolist(), a.tolist())) != dict(zip(rk.tolist(), ra.tolist())):
                bad.append((t, "state"))
            if sh.peak() != ref.peak():
                bad.append((t, "peak"))
            if bad:
                break
        out.put((rank, bad, sh.retained_mass() == ref.retained_mass(), list(sh.glob), most))
    finally:
        dist.destroy_process_group()


def _circuit(C, case):
    if case["kind"] == "mix":
        return C.random_mix_circuit(case["n"], case["gates"], seed=case["seed"], sigma=0.05, K=case["K"], p=case["p"])
    return C.brickwork_circuit(case["n"], case["layers"], seed=case["seed"], sigma=0.05, K=case["K"], p=case["p"])


@pytest.mark.parametrize("world,case", [
    (2, {"kind": "mix", "n": 10, "gates": 24, "seed": 41, "K": 150, "p": 0.999, "prec": 0}),
    (2, {"kind": "brick", "n": 10, "layers": 2, "seed": 42, "K": 64, "p": 1.0, "prec": 1}),
    (4, {"kind": "mix", "n": 9, "gates": 20, "seed": 43, "K": 100, "p": 0.99, "prec": 0}),
])
def test_sharded_state_equals_the_oracle_alone(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, bad, same_F, glob, n_local in sorted(res):
        assert not bad, (rank, bad[:3])
        assert same_F
        assert n_local > 0  # the exchanges spread the terms over every rank at some point
    assert len({tuple(r[3]) for r in res}) == 1  # every rank agrees on the partition qubits
    g = world.bit_length() - 1
    assert res[0][3] != list(range(case["n"] - g, case["n"]))  # gates on partition qubits swapped them out


def test_single_rank_is_the_plain_state(oracle_mod):
    """Without a process group the sharded state is one partition: the same
    result as the oracle, the same orchestration code."""
    sys.path.insert(0, ROOT)
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300.shard import ShardedState
    c = C.random_mix_circuit(9, 16, seed=5, sigma=0.05, K=80, p=0.995)
    sh = ShardedState(c.n, c.K, c.p, lambda n: OracleEngine(oracle_mod, n))
    ref = oracle_mod.Oracle(c.n, c.K, c.p)
    for q, u in c.gates:
        sh.apply_gate(q, u)
        ref.apply_gate(q, u)
        assert sh.truncate() == ref.truncate()
    k, a = sh.export()
    rk, ra, _ = ref.export()
    assert dict(zip(k.tolist(), a.tolist())) == dict(zip(rk.tolist(), ra.tolist()))
    assert sh.peak() == ref.peak()
