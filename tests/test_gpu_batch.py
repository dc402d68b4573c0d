"""Batched form (svb_*): many circuits of uneven n, K and length advanced
together in one segmented state must each give exactly the result of the
oracle run on that circuit alone (same gates, same per-gate top-k)."""
import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C
from tests.parity import batched_sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import sv as _sv
    _sv.load_library()
    return _sv


def _as_dict(keys, amps):
    return {int(k): complex(a) for k, a in zip(keys, amps)}


def _check_slot(b, slot, orc, what):
    gk, ga = b.export(slot)
    ok, oa, _ = orc.export()
    g, o = _as_dict(gk, ga), _as_dict(ok, oa)
    assert g.keys() == o.keys(), f"{what}: key sets differ ({len(g)} vs {len(o)})"
    bad = [k for k in g if g[k] != o[k]]
    assert not bad, f"{what}: {len(bad)} amplitudes differ"
    assert b.peak(slot) == orc.peak(), what
    assert b.retained_mass(slot) == orc.retained_mass(), what


def _circuits(rng, count):
    out = []
    for j in range(count):
        n = int(rng.integers(10, 31))
        depth = int(rng.integers(1, 4))
        K = 1 << int(rng.integers(6, 13))
        out.append(C.brickwork_circuit(n, depth, seed=int(rng.integers(1 << 30)), sigma=0.05, K=K, p=1.0))
    return out


@pytest.mark.parametrize("layer", [True, False], ids=["one_launch", "kernels"])
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_oracle_per_circuit(sv, oracle_mod, prec, layer):
    """Both forms of the step (the persistent one-launch layer kernel and the
    separate kernels) against the oracle, circuit by circuit."""
    rng = np.random.default_rng(31 + prec)
    circs = _circuits(rng, 10)
    b = sv.Batch(16, prec=prec)
    b.set_layer_kernel(layer)
    slots = [b.add(c.n, c.K) for c in circs]
    orcs = [oracle_mod.Oracle(c.n, c.K, 1.0, prec=prec) for c in circs]
    pos = [0] * len(circs)
    done = [False] * len(circs)
    step = 0
    while not all(done):
        gates = []
        for j, c in enumerate(circs):
            if done[j]:
                continue
            # every third step circuit j sits out once (identity pass-through)
            if (step + j) % 3 == 0 and pos[j] > 0 and pos[j] % 2 == 1:
                continue
            q, u = c.gates[pos[j]]
            gates.append((slots[j], q, u))
            orcs[j].apply_gate(q, u)
            orcs[j].truncate()
            pos[j] += 1
        b.step(gates)
        for j, c in enumerate(circs):
            if not done[j] and pos[j] == len(c.gates):
                _check_slot(b, slots[j], orcs[j], f"circuit {j} (n={c.n}, K={c.K})")
                b.remove(slots[j])
                done[j] = True
        step += 1
    b.step([])  # drops the retired slots
    b.close()


@pytest.mark.parametrize("layer", [True, False], ids=["one_launch", "kernels"])
def test_batch_slot_reuse_and_late_arrivals(sv, oracle_mod, layer):
    rng = np.random.default_rng(7)
    circs = _circuits(rng, 8)
    b = sv.Batch(4, prec=1)
    b.set_layer_kernel(layer)
    live = {}  # slot -> (circuit index, position, oracle)
    queue = list(range(len(circs)))
    finished = 0
    while finished < len(circs):
        while queue and len(live) < 4:
            j = queue.pop(0)
            c = circs[j]
            s = b.add(c.n, c.K)
            assert s not in live
            live[s] = [j, 0, oracle_mod.Oracle(c.n, c.K, 1.0, prec=1)]
        gates = []
        for s, (j, p, o) in live.items():
            q, u = circs[j].gates[p]
            gates.append((s, q, u))
            o.apply_gate(q, u)
            o.truncate()
            live[s][1] += 1
        b.step(gates)
        for s in list(live):
            j, p, o = live[s]
            if p == len(circs[j].gates):
                _check_slot(b, s, o, f"circuit {j}")
                b.remove(s)
                del live[s]
                finished += 1
        b.step([])  # frees the retired slots for the next arrivals
    b.close()


@pytest.mark.parametrize("layer", [True, False], ids=["one_launch", "kernels"])
def test_pipelined_readout_after_removal(sv, oracle_mod, layer):
    """Slots retired with svb_peak_async and removed at once, their readouts
    collected after later steps (and adds into the freed slots) have been
    enqueued: each gives the oracle's peak and retained mass."""
    rng = np.random.default_rng(19)
    circs = _circuits(rng, 9)
    b = sv.Batch(3, prec=0)
    b.set_layer_kernel(layer)
    live, queue, tickets, want = {}, list(range(len(circs))), [], {}
    while queue or live:
        while queue and len(live) < 3:
            j = queue.pop(0)
            s = b.add(circs[j].n, circs[j].K)
            live[s] = [j, 0, oracle_mod.Oracle(circs[j].n, circs[j].K, 1.0, prec=0)]
        gates = []
        for s, (j, p, o) in live.items():
            q, u = circs[j].gates[p]
            gates.append((s, q, u))
            o.apply_gate(q, u)
            o.truncate()
            live[s][1] += 1
        b.step(gates)
        for s in list(live):
            j, p, o = live[s]
            if p == len(circs[j].gates):
                tickets.append((j, b.peak_async(s)))
                want[j] = (o.peak(), o.retained_mass())
                b.remove(s)
                del live[s]
        b.step([])
    assert len(tickets) == len(circs)
    for j, t in tickets:
        key, prob, f = b.peak_wait(t)
        assert (key, prob) == want[j][0], f"circuit {j}"
        assert f == want[j][1], f"circuit {j}"
    with pytest.raises(sv.SVError):
        b.peak_wait(tickets[0][1])  # collected once
    b.close()


def test_batch_argument_errors(sv):
    b = sv.Batch(2, prec=1)
    s = b.add(8, 64)
    with pytest.raises(sv.SVError):
        b.add(64, 4)                       # n above 63
    with pytest.raises(sv.SVError):
        sv.svb_add(b.h, 8, 16, 0.9)        # p-mass not offered in the batched form
    with pytest.raises(sv.SVError):
        b.step([(s, (0, 0), np.eye(4))])  # repeated qubit
    with pytest.raises(sv.SVError):
        b.step([(s, (9,), np.eye(2))])     # qubit above n
    with pytest.raises(sv.SVError):
        b.step([(1, (0,), np.eye(2))])     # slot not in use
    b.step([(s, (0,), C.mat_h())])
    assert b.num_terms(s) == 2
    b.close()


def test_batch_sort_key_bit_bound(sv):
    """n plus the slot-index bits must fit the 64-bit sort key: n = 56 fits
    while the highest slot in use is below 255, and not after."""
    b = sv.Batch(400, prec=1)
    big = b.add(56, 16)
    assert big == 0
    small = [b.add(8, 16) for _ in range(254)]  # slots 1..254: top = 255, 8 bits
    with pytest.raises(sv.SVError):
        b.add(8, 16)                       # slot 255 would need a ninth bit
    b.remove(big)
    b.step([])                             # frees slot 0
    with pytest.raises(sv.SVError):
        b.add(57, 16)                      # 57 + 8 bits
    s = b.add(56, 16)                      # lowest free slot is 0 again
    assert s == 0
    b.step([(s, (55,), C.mat_h())] + [(t, (0,), C.mat_h()) for t in small[:3]])
    assert b.num_terms(s) == 2 and b.num_terms(small[0]) == 2 and b.num_terms(small[5]) == 1
    keys, _ = b.export(s)
    assert sorted(int(k) for k in keys) == [0, 1 << 55]
    b.close()


def _run_batch(sv, circs, tune, graphs, reps=1, layer=False):
    b = sv.Batch(16, prec=1)
    b.set_autotune(tune)
    b.set_graphs(graphs)
    b.set_layer_kernel(layer)
    slots = [b.add(c.n, c.K) for c in circs]
    longest = max(len(c.gates) for c in circs)
    for _ in range(reps):
        for g in range(longest):
            b.step([(slots[j], *c.gates[g]) for j, c in enumerate(circs) if g < len(c.gates)])
    res = [(b.export(s), b.peak(s), b.retained_mass(s)) for s in slots]
    stats = (b.autotune_stats(), b.graph_stats())
    b.close()
    return res, stats


def _same(ra, rb):
    for (ea, pa, fa), (eb, pb, fb) in zip(ra, rb):
        assert _as_dict(*ea) == _as_dict(*eb)
        assert pa == pb and fa == fb


def test_autotuned_shapes_give_identical_results(sv):
    """The autotuner runs every candidate launch shape on live steps; the
    result of every circuit must be the same as with the fixed shapes."""
    circs = _circuits(np.random.default_rng(71), 8)
    fixed, (tstats, _) = _run_batch(sv, circs, tune=False, graphs=False)
    tuned, (tstats2, _) = _run_batch(sv, circs, tune=True, graphs=False)
    assert tstats["trials"] == 0
    assert tstats2["trials"] > 0 and tstats2["classes"] > 0
    _same(fixed, tuned)
    # the one-launch step tunes its blocks per SM (timings read two steps on)
    layer, (tstats3, _) = _run_batch(sv, circs, tune=True, graphs=True, layer=True)
    assert tstats3["trials"] > 0 and tstats3["classes"] > 0
    _same(fixed, layer)


def test_graph_replay_gives_identical_results(sv):
    """Circuits held at their K repeat the same step sizes, so the captured
    graphs are replayed; results must equal direct launches."""
    rng = np.random.default_rng(72)
    circs = [C.brickwork_circuit(20, 3, seed=int(rng.integers(1 << 30)), sigma=0.05, K=64, p=1.0)
             for _ in range(5)]
    direct, _ = _run_batch(sv, circs, tune=False, graphs=False)
    graphed, (_, gstats) = _run_batch(sv, circs, tune=False, graphs=True)
    assert gstats["captures"] >= 1 and gstats["launches"] > gstats["captures"]
    _same(direct, graphed)
    tuned, (tstats, gstats2) = _run_batch(sv, circs, tune=True, graphs=True)
    _same(direct, tuned)


def test_layer_kernel_graphs_and_separate_kernels_agree(sv):
    """The one-launch step, direct and replayed from its graph, equals the
    separate kernels bit for bit; steps of circuits held at their K replay
    the captured launch."""
    rng = np.random.default_rng(73)
    circs = [C.brickwork_circuit(24, 3, seed=int(rng.integers(1 << 30)), sigma=0.05, K=256, p=1.0)
             for _ in range(6)]
    kernels, _ = _run_batch(sv, circs, tune=False, graphs=False, layer=False)
    direct, (_, g0) = _run_batch(sv, circs, tune=False, graphs=False, layer=True)
    graphed, (_, g1) = _run_batch(sv, circs, tune=False, graphs=True, layer=True)
    assert g0["launches"] == 0
    assert g1["captures"] >= 1 and g1["launches"] > 2 * g1["captures"]
    _same(kernels, direct)
    _same(kernels, graphed)


@pytest.mark.parametrize("layer", [True, False], ids=["one_launch", "kernels"])
def test_complex64_batch_against_complex128_oracle(sv, oracle_mod, layer):
    """Circuits of the 512-circuit batched workload, advanced together in
    complex64: each slot equals the complex64 oracle exactly and stays within
    2e-6 per amplitude of the complex128 oracle, with the same kept terms and
    the same peak string."""
    sample = batched_sample()
    circs = [c for _, c in sample]
    b = sv.Batch(len(circs), prec=1)
    b.set_layer_kernel(layer)
    slots = [b.add(c.n, c.K) for c in circs]
    o64 = [oracle_mod.Oracle(c.n, c.K, 1.0, prec=1) for c in circs]
    o128 = [oracle_mod.Oracle(c.n, c.K, 1.0, prec=0) for c in circs]
    for t in range(max(len(c.gates) for c in circs)):
        gates = []
        for s, c, x, y in zip(slots, circs, o64, o128):
            if t < len(c.gates):
                q, u = c.gates[t]
                gates.append((s, q, u))
                for o in (x, y):
                    o.apply_gate(q, u)
                    o.truncate()
        b.step(gates)
    for (j, c), s, x, y in zip(sample, slots, o64, o128):
        what = f"circuit {j} (n={c.n}, K={c.K})"
        _check_slot(b, s, x, what)
        gk, ga = b.export(s)
        wk, wa, _ = y.export()
        g, w = _as_dict(gk, ga), _as_dict(wk, wa)
        assert g.keys() == w.keys(), what
        d = max(abs(g[k] - w[k]) for k in w)
        assert d <= 2e-6, f"{what}: max |d amp| {d:.3e}"
        assert b.peak(s)[0] == y.peak()[0], what
    b.close()
