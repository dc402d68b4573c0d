"""Host logic of the serving loop, run against a fake batch on the CPU:
admission in arrival order within the slot and byte budgets, one gate per
resident circuit per step, retirement right after a circuit's last gate, and
the latency bookkeeping."""
import numpy as np
import pytest

from paper_2607_07816_b300 import serve


class FakeCircuit:
    def __init__(self, n, K, lengths_m):
        self.n = n
        self.K = K
        self.gates = [(tuple(range(m)), np.eye(1 << m)) for m in lengths_m]


class FakeBatch:
    """Records the calls the loop makes and checks the batch's own rules."""

    def __init__(self, max_slots):
        self.max_slots = max_slots
        self.state = {}  # slot -> "used" | "removing"
        self.applied = {}  # slot -> gates applied
        self.steps = []
        self.adds = []

    def add(self, n, K):
        free = [s for s in range(self.max_slots) if s not in self.state]
        assert free, "add with no free slot"
        s = free[0]
        self.state[s] = "used"
        self.applied[s] = 0
        self.adds.append((n, K, s))
        return s

    def remove(self, slot):
        assert self.state.get(slot) == "used"
        self.state[slot] = "removing"

    def step(self, gates):
        slots = [g[0] for g in gates]
        assert len(set(slots)) == len(slots)
        for s in slots:
            assert self.state.get(s) == "used"
            self.applied[s] += 1
        for s in [s for s, v in self.state.items() if v == "removing"]:
            del self.state[s]
        self.steps.append(sorted(slots))

    def step_table(self, table):
        self.step([(int(r["slot"]), tuple(int(x) for x in r["q"][:int(r["m"])]), None) for r in table])

    def peak(self, slot):
        return (self.applied[slot], 0.5)

    def peak_async(self, slot):
        assert self.state.get(slot) == "used", "readout of a slot not in use"
        if not hasattr(self, "tickets"):
            self.tickets = {}
        t = len(self.tickets)
        self.tickets[t] = self.applied[slot]
        return t

    def peak_wait(self, ticket):
        assert ticket in self.tickets, "ticket collected twice or never issued"
        return (self.tickets.pop(ticket), 0.5, 1.0)

    def retained_mass(self, slot):
        return 1.0

    def export(self, slot):
        return np.zeros(0, np.uint64), np.zeros(0)


def test_footprint_and_slot_limit():
    c = FakeCircuit(10, 1000, [1, 2, 3])
    assert serve.footprint(c) == 1000 * 8 * 16
    assert serve.slot_limit(54, 1023) == 1023
    assert serve.slot_limit(56, 1023) == 255
    assert serve.slot_limit(63, 1023) == 1


def test_saturated_run_respects_budgets():
    rng = np.random.default_rng(0)
    circs = [FakeCircuit(8, int(rng.integers(1, 5)) * 100, [2] * int(rng.integers(1, 9))) for _ in range(40)]
    budget = 4 * 100 * 4 * 16 * 3  # a few requests at a time
    fb = FakeBatch(6)
    srv = serve.Server(budget, max_slots=6, batch=fb)
    res = srv.run(circs, clock=lambda: srv.steps)
    assert len(res) == 40
    for r, c in zip(res, circs):
        assert r.peak_key == len(c.gates)  # every gate of the circuit was applied once
    assert srv.peak_bytes <= budget
    assert srv.peak_resident <= 6
    assert max(len(s) for s in fb.steps) <= 6
    # admission follows arrival order (all at 0: input order)
    admitted = sorted(range(40), key=lambda j: (res[j].admitted, j))
    assert admitted == list(range(40))


def test_arrivals_wait_and_overlap():
    circs = [FakeCircuit(8, 10, [1] * L) for L in (10, 3, 3, 4, 1)]
    arrivals = [0, 2, 2, 5, 20]
    fb = FakeBatch(8)
    srv = serve.Server(1 << 40, max_slots=8, batch=fb)
    res = srv.run(circs, arrivals=arrivals, clock=lambda: srv.steps + (100 if fb.steps and not fb.state else 0))
    for r, a in zip(res, arrivals):
        assert r.admitted >= a
    # request 1 and 2 run while request 0 is resident (continuous batching);
    # a readout is collected once the next step is enqueued (request 1's last
    # gate is step 5), or at once when no step follows (request 0's is step 10)
    assert res[1].admitted < res[0].finished and res[2].admitted < res[0].finished
    assert res[1].admitted == 2 and res[1].finished == 6
    assert res[0].finished == 10
    assert all(r.peak_key == len(c.gates) for r, c in zip(res, circs))


def test_oversized_request_runs_alone():
    circs = [FakeCircuit(8, 1000, [2] * 3), FakeCircuit(8, 10 ** 6, [2] * 2), FakeCircuit(8, 1000, [2] * 3)]
    fb = FakeBatch(8)
    srv = serve.Server(1000 * 4 * 16 * 2, max_slots=8, batch=fb)
    res = srv.run(circs, clock=lambda: srv.steps)
    # request 1 does not fit beside request 0; it waits until request 0 has
    # run its last step and left, then runs alone (readouts are collected a
    # step later, so admission is compared with the steps each request ran)
    assert res[1].admitted >= len(circs[0].gates)
    assert all(len(s) == 1 for s in fb.steps[3:5])
    assert res[2].admitted >= res[1].admitted + len(circs[1].gates)


def test_fifo_latencies_and_percentiles():
    lat = serve.fifo_latencies([0.0, 0.5, 10.0], [1.0, 1.0, 2.0])
    assert np.allclose(lat, [1.0, 1.5, 2.0])
    res = [serve.Result(j, 0, 1.0, 1.0, 0.0, 0.0, float(j + 1)) for j in range(100)]
    p50, p99 = serve.percentiles(res)
    assert p50 == pytest.approx(50.5) and p99 == pytest.approx(99.01)
    t = serve.poisson_arrivals(20000, 50.0, 1)
    assert np.all(np.diff(t) > 0)
    assert 20000 / t[-1] == pytest.approx(50.0, rel=0.03)


class FakeState:
    """Stands in for a single-state handle on the CPU: counts gates."""
    made = []

    def __init__(self, n, K, p, prec=0, stream=0):
        self.n, self.K, self.stream = n, K, stream
        self.gates = 0
        FakeState.made.append(self)

    def apply_gate(self, q, u):
        self.gates += 1

    def truncate(self):
        return (self.K, 1.0)

    def peak(self):
        return (1000 + self.gates, 0.25)

    def retained_mass(self):
        return 0.5

    def export(self):
        return np.zeros(0, np.uint64), np.zeros(0)

    def close(self):
        pass


class FakeStream:
    cuda_stream = 7


def test_large_requests_run_solo_beside_the_batch(monkeypatch):
    monkeypatch.setattr(serve.sv, "SparseState", FakeState)
    FakeState.made = []
    circs = [FakeCircuit(8, 100, [2] * 4), FakeCircuit(8, 1 << 20, [2] * 6), FakeCircuit(8, 100, [2] * 3),
             FakeCircuit(8, 1 << 21, [1] * 5)]
    fb = FakeBatch(8)
    srv = serve.Server(1 << 40, max_slots=8, batch=fb, solo_min_terms=1 << 20, solo_stream=FakeStream)
    res = srv.run(circs)
    assert srv.solo_served == 2
    assert [s.K for s in FakeState.made] == [1 << 20, 1 << 21]
    assert all(s.stream == 7 for s in FakeState.made)
    # solo requests: every gate on their own handle; batched ones: in the batch's steps
    assert res[1].peak_key == 1006 and res[3].peak_key == 1005
    assert res[0].peak_key == 4 and res[2].peak_key == 3
    assert sorted(s for _, _, s in fb.adds) == [0, 1]
    assert all(r.finished >= r.admitted for r in res)


def test_solo_requests_share_the_budget(monkeypatch):
    monkeypatch.setattr(serve.sv, "SparseState", FakeState)
    FakeState.made = []
    big = FakeCircuit(8, 1 << 20, [2] * 2)
    small = FakeCircuit(8, 100, [2] * 2)
    budget = serve.footprint(big) + serve.footprint(small) // 2
    fb = FakeBatch(8)
    srv = serve.Server(budget, max_slots=8, batch=fb, solo_min_terms=1 << 20, solo_stream=FakeStream)
    res = srv.run([big, small])
    # the small request does not fit beside the solo one: admitted after it finished
    assert res[1].admitted >= res[0].finished
    assert srv.peak_bytes <= budget
