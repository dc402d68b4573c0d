"""CUDA path (through the C ABI) against the CPU oracle, element by element.

With the same operation order on both sides (fused multiply-adds in
ascending input order, exact fixed-point masses, correctly rounded sqrt and
division), the kept key sets and the amplitudes are expected to be identical,
so these tests compare exactly.  They cover several tiles with ragged tails,
every gate width m = 1..4, exact ties in probability, p-cuts landing on a
prefix sum, top-k and p-mass together, and both precisions.
"""
import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C
from tests.parity import assert_states_equal, run_both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import sv as _sv
    _sv.load_library()
    return _sv


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_mirror_n12(sv, oracle_mod, prec):
    c = C.exact_mirror_n12()
    g = sv.SparseState(c.n, c.K, c.p, prec=prec)
    o = oracle_mod.Oracle(c.n, c.K, c.p, prec=prec)
    run_both(c.gates, g, o)
    key, pr = g.peak()
    assert key == c.hidden
    assert pr > 1.0 - (1e-12 if prec == 0 else 1e-5)


@pytest.mark.parametrize("seed", range(8))
def test_random_gates_topk_and_pmass(sv, oracle_mod, seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(6, 21))
    K = int(rng.choice([7, 100, 1000, 5000, 1 << 20]))
    p = float(rng.choice([1.0, 0.999, 0.95, 0.5]))
    prec = int(seed % 2)
    gates = []
    for _ in range(24):
        m = int(rng.integers(1, min(4, n) + 1))
        kind = str(rng.choice(["haar", "haar", "mcx", "h"]))
        gates.append(C.random_gate(n, m, rng, kind))
    g = sv.SparseState(n, K, p, prec=prec)
    o = oracle_mod.Oracle(n, K, p, prec=prec)
    run_both(gates, g, o)


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_multi_tile_states(sv, oracle_mod, prec):
    """Loaded states of 1..~70k terms on 30 qubits: many sort and
    compaction tiles, ragged tails, all gate widths."""
    rng = np.random.default_rng(77 + prec)
    for count in [1, 2, 1023, 4097, 9000, 70001]:
        n = 30
        keys, amps = C.random_state(n, count, rng)
        K = max(1, count // 3)
        g = sv.SparseState(n, K, 0.97, prec=prec)
        o = oracle_mod.Oracle(n, K, 0.97, prec=prec)
        g.load(keys, amps)
        o.load(keys, amps)
        assert_states_equal(g, o, what=f"load {count}")
        gates = [C.random_gate(n, m, rng, "haar") for m in (1, 2, 3, 4)]
        run_both(gates, g, o)


def test_equal_probabilities_cut_by_key(sv, oracle_mod):
    n = 12
    for K in [1, 5, 1000, 4095]:
        g = sv.SparseState(n, K, 1.0)
        o = oracle_mod.Oracle(n, K, 1.0)
        gates = [((i,), C.mat_h()) for i in range(n)]
        for (q, u) in gates:
            g.apply_gate(q, u)
            o.apply_gate(q, u)
        assert g.num_terms() == 1 << n
        assert g.peak() == o.peak()  # read from the state (no truncation yet)
        assert g.truncate() == o.truncate()
        assert g.peak() == o.peak()  # reduced from the compaction's per-block partials
        assert_states_equal(g, o, what=f"K={K}")


@pytest.mark.parametrize("prec", [0, 1])
def test_peak_ties_across_many_compaction_blocks(sv, oracle_mod, prec):
    """2^20 equal probabilities cut to K: the peak after the truncation is the
    smallest kept key, found among the partial results of many blocks; after
    one more gate the peak is read from the state again."""
    n = 20
    for K in [(1 << 19) + 12345, 3]:
        g = sv.SparseState(n, K, 1.0, prec=prec)
        o = oracle_mod.Oracle(n, K, 1.0, prec=prec)
        for i in range(n):
            g.apply_gate((i,), C.mat_h())
            o.apply_gate((i,), C.mat_h())
        assert g.truncate() == o.truncate()
        assert g.peak() == o.peak()
        g.apply_gate((3, 11), C.mat_cz())
        o.apply_gate((3, 11), C.mat_cz())
        assert g.peak() == o.peak()


def test_p_cut_on_exact_prefix_and_forced_ties(sv, oracle_mod):
    keys = np.array([5, 9, 2, 7, 11, 3], dtype=np.uint64)
    amps = np.array([0.5 + 0.5j, 0.5, 0.25 + 0.25j, -0.25 + 0.25j, 0.0625, 0.0625j])
    for p in [0.75, 0.75 + 1e-12, 0.5, 0.875, 0.999, 1e-300]:
        for K in [1, 3, 100]:
            g = sv.SparseState(4, K, p)
            o = oracle_mod.Oracle(4, K, p)
            g.load(keys, amps)
            o.load(keys, amps)
            assert g.truncate() == o.truncate(), (p, K)
            assert_states_equal(g, o, what=f"p={p} K={K}")


def test_tied_random_states(sv, oracle_mod):
    rng = np.random.default_rng(11)
    for trial in range(6):
        keys, amps = C.random_state(24, 20000, rng, ties=True)
        K = int(rng.integers(1, 20000))
        p = float(rng.uniform(0.3, 1.0))
        g = sv.SparseState(24, K, p)
        o = oracle_mod.Oracle(24, K, p)
        g.load(keys, amps)
        o.load(keys, amps)
        assert g.truncate() == o.truncate()
        assert g.peak() == o.peak()
        assert_states_equal(g, o, what=f"trial {trial}")


def test_structured_gates_keep_count(sv, oracle_mod):
    rng = np.random.default_rng(5)
    keys, amps = C.random_state(20, 3000, rng)
    g = sv.SparseState(20)
    g.load(keys, amps)
    for m in (2, 3, 4):
        for _ in range(3):
            qs = tuple(int(x) for x in rng.choice(20, size=m, replace=False))
            g.apply_gate(qs, C.mat_mcx(m))
            assert g.num_terms() == 3000
    g.apply_gate((0, 19), C.mat_cz())
    assert g.num_terms() == 3000


def test_random_mix_circuit_n60(sv, oracle_mod):
    c = C.random_mix_circuit(60, 60, seed=9, sigma=0.05, K=2000, p=0.9999)
    for prec in (0, 1):
        g = sv.SparseState(c.n, c.K, c.p, prec=prec)
        o = oracle_mod.Oracle(c.n, c.K, c.p, prec=prec)
        run_both(c.gates, g, o, check_every=False)


def test_brickwork_n40_reduced_K(sv, oracle_mod):
    c = C.brickwork_n40(layers=3, K=1 << 12)
    g = sv.SparseState(c.n, c.K, c.p)
    o = oracle_mod.Oracle(c.n, c.K, c.p)
    run_both(c.gates, g, o, check_every=False)


def test_pipelined_peak_readout_matches_oracle_gate_by_gate(sv, oracle_mod):
    # every gate's peak is enqueued and read back later (up to 8 in flight);
    # each must be the peak the oracle has after that gate
    c = C.brickwork_n40(layers=3, K=1 << 10)
    g = sv.SparseState(c.n, c.K, c.p)
    o = oracle_mod.Oracle(c.n, c.K, c.p)
    tickets, expected, got = [], [], []
    for q, u in c.gates:
        g.apply_gate(q, u)
        g.truncate()
        o.apply_gate(q, u)
        o.truncate()
        tickets.append(g.peak_async())
        expected.append(o.peak())
        if len(tickets) - len(got) == 8:
            got.append(g.peak_wait(tickets[len(got)]))
    while len(got) < len(tickets):
        got.append(g.peak_wait(tickets[len(got)]))
    assert got == expected
    assert g.peak() == expected[-1]
    # a ticket whose slot was reused, or one never issued, is rejected
    with pytest.raises(sv.SVError) as e:
        g.peak_wait(tickets[0])
    assert e.value.status == sv.SV_E_ARG
    with pytest.raises(sv.SVError) as e:
        g.peak_wait(tickets[-1] + 1)
    assert e.value.status == sv.SV_E_ARG
    # the handle stays usable, and an emptied state has no peak to enqueue
    assert g.peak_wait(g.peak_async()) == expected[-1]
    g.load(np.zeros(0, dtype=np.uint64), np.zeros(0))
    with pytest.raises(sv.SVError) as e:
        g.peak_async()
    assert e.value.status == sv.SV_E_STATE


def test_complex64_close_to_complex128(sv, oracle_mod):
    c = C.brickwork_circuit(16, 4, seed=3, sigma=0.05, K=1 << 10, p=1.0)
    g64 = sv.SparseState(c.n, c.K, c.p, prec=1)
    o128 = oracle_mod.Oracle(c.n, c.K, c.p, prec=0)
    g64.run(c.gates)
    o128.run(c.gates)
    assert g64.peak()[0] == o128.peak()[0]
    gk, ga = g64.export()
    ok, oa, _ = o128.export()
    common, gi, oi = np.intersect1d(gk, ok, return_indices=True)
    assert len(common) > 0.9 * len(ok)
    assert np.max(np.abs(ga[gi] - oa[oi])) <= 2e-6


def test_argument_errors(sv):
    g = sv.SparseState(5)
    with pytest.raises(sv.SVError) as e:
        g.apply_gate((0, 0), np.eye(4))
    assert e.value.status == sv.SV_E_ARG
    with pytest.raises(sv.SVError) as e:
        g.apply_gate((7,), np.eye(2))
    assert e.value.status == sv.SV_E_ARG
    with pytest.raises(sv.SVError) as e:
        g.apply_gate((1,), np.array([[1, 1], [0, 1]]))
    assert e.value.status == sv.SV_E_NOT_UNITARY
    with pytest.raises(sv.SVError) as e:
        g.load(np.array([1, 1], dtype=np.uint64), np.array([0.6, 0.8]))
    assert e.value.status == sv.SV_E_ARG
    with pytest.raises(sv.SVError) as e:
        g.load(np.array([32], dtype=np.uint64), np.array([1.0]))
    assert e.value.status == sv.SV_E_ARG
    # the handle is still usable after rejected arguments
    g.apply_gate((1,), C.mat_h())
    assert g.num_terms() == 2


def test_probs_dump_and_export_roundtrip(sv, oracle_mod):
    rng = np.random.default_rng(3)
    keys, amps = C.random_state(33, 5000, rng, ties=True)
    g = sv.SparseState(33, prec=0)
    o = oracle_mod.Oracle(33)
    g.load(keys, amps)
    o.load(keys, amps)
    pk, pp = g.probs()
    ok, _, op = o.export()
    assert np.array_equal(pk, ok)
    assert np.array_equal(pp, op)
    ek, ea = g.export()
    g2 = sv.SparseState(33)
    g2.load(ek, ea)
    assert_states_equal(g2, o, what="reload")


def test_exact_cancellation_drops_zero_terms(sv, oracle_mod):
    """H on every qubit twice: the second layer cancels all but one term
    exactly, so the library must drop exact zeros (Sec. IV-A)."""
    n = 14
    for prec in (0, 1):
        g = sv.SparseState(n, prec=prec)
        o = oracle_mod.Oracle(n, prec=prec)
        gates = [((i,), C.mat_h()) for i in range(n)] + [((i,), C.mat_h()) for i in reversed(range(n))]
        run_both(gates, g, o, truncate=False, check_every=False)
        assert g.num_terms() == o.num_terms()


def test_skewed_keys_large_state(sv, oracle_mod):
    """Most keys share their high bits, a few stand apart: a state far larger
    than one shared-memory batch, with strongly skewed bit patterns, goes
    through the sorted path with the oracle's result."""
    rng = np.random.default_rng(123)
    n = 30
    low = rng.choice(1 << 20, size=30000, replace=False).astype(np.uint64)
    high = (rng.choice(1 << 10, size=200, replace=False).astype(np.uint64) << np.uint64(20)) | np.uint64(7)
    keys = np.unique(np.concatenate([low, high]))
    amps = (rng.standard_normal(len(keys)) + 1j * rng.standard_normal(len(keys)))
    amps /= np.linalg.norm(amps)
    g = sv.SparseState(n, 1 << 20, 1.0)
    o = oracle_mod.Oracle(n, 1 << 20, 1.0)
    g.load(keys, amps)
    o.load(keys, amps)
    gates = [C.random_gate(n, 2, rng, "haar") for _ in range(3)]
    gates += [((0, 1), C.haar_unitary(4, rng)), ((2, 3), C.haar_unitary(4, rng)), ((4,), C.mat_h())]
    run_both(gates, g, o)


@pytest.mark.parametrize("prec", [0, 1])
def test_brickwork_local_and_global_gates(sv, oracle_mod, prec):
    """Small states (the first gates) take the shared-memory kernel, larger
    ones the sorted path; the result is the oracle's either way."""
    c = C.brickwork_circuit(24, 6, seed=77, sigma=0.05, K=1 << 14, p=1.0)
    g = sv.SparseState(c.n, c.K, c.p, prec=prec)
    o = oracle_mod.Oracle(c.n, c.K, c.p, prec=prec)
    run_both(c.gates, g, o, check_every=False)
    st = g.stats()
    assert st["local_gates"] > 0 and st["global_gates"] > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_ring_u3cz_reordered_and_fused(sv, oracle_mod, prec):
    """The ring-connected u3/cz workload after reordering and fusion into
    two-qubit blocks (one update and one truncation per block), GPU against
    the oracle on the same block list."""
    from paper_2607_07816_b300 import fusion, qasm
    c = qasm.sharp_peak_circuit(n=44, blocks=93, K=32)
    blocks = fusion.prepare(c.gates, 2)
    g = sv.SparseState(c.n, c.K, 1.0, prec=prec)
    o = oracle_mod.Oracle(c.n, c.K, 1.0, prec=prec)
    run_both(blocks, g, o, check_every=False)
    gq = sv.SparseState(c.n, 1 << 12, 1.0, prec=prec)
    oq = oracle_mod.Oracle(c.n, 1 << 12, 1.0, prec=prec)
    run_both(fusion.fuse(c.gates, 4), gq, oq, check_every=False)


@pytest.mark.parametrize("prec", [0, 1])
def test_expand_first_variant_matches_oracle_and_group_first(sv, oracle_mod, prec):
    """The paper's expand-first formulation gives the oracle's result bit for
    bit, and the same storage order as the group-first path."""
    rng = np.random.default_rng(640 + prec)
    for trial in range(3):
        n = int(rng.integers(8, 30))
        K = int(rng.choice([50, 3000, 1 << 16]))
        gates = [C.random_gate(n, int(rng.integers(1, 5)) if n >= 4 else 1, rng,
                               str(rng.choice(["haar", "mcx", "h"]))) for _ in range(16)]
        e = sv.SparseState(n, K, 1.0, prec=prec)
        e.set_variant(1)
        o = oracle_mod.Oracle(n, K, 1.0, prec=prec)
        run_both(gates, e, o)
        g = sv.SparseState(n, K, 1.0, prec=prec)
        g.run(gates)
        ek, ea = e.export()
        gk, ga = g.export()
        assert np.array_equal(ek, gk) and np.array_equal(ea, ga)
    with pytest.raises(sv.SVError):
        e.set_variant(3)


@pytest.mark.parametrize("prec", [0, 1])
def test_radix_grouping_variant_matches_merge_grouping(sv, oracle_mod, prec):
    """Grouping by a full radix sort (variant 2) and by partition and merge
    (the default) give the oracle's result and the same storage order, on
    gates of every width, over states large enough for many merge tiles."""
    rng = np.random.default_rng(650 + prec)
    for trial in range(3):
        n = int(rng.integers(20, 41))
        K = int(rng.choice([5000, 1 << 15, 1 << 16]))
        gates = [C.random_gate(n, int(rng.integers(1, 5)), rng, str(rng.choice(["haar", "mcx", "h"])))
                 for _ in range(20)]
        a = sv.SparseState(n, K, 1.0, prec=prec)
        a.set_variant(2)
        o = oracle_mod.Oracle(n, K, 1.0, prec=prec)
        run_both(gates, a, o, check_every=False)
        b = sv.SparseState(n, K, 1.0, prec=prec)
        b.run(gates)
        ak, aa = a.export()
        bk, ba = b.export()
        assert np.array_equal(ak, bk) and np.array_equal(aa, ba)


def test_handles_release_device_memory(sv):
    """Creating, using and destroying handles (plain and batched) returns
    their device memory: the free memory after many cycles matches the
    free memory after the first (allocator caches aside, nothing grows)."""
    import torch
    c = C.brickwork_circuit(22, 2, seed=9, sigma=0.05, K=1 << 14, p=0.99)

    def cycle():
        g = sv.SparseState(c.n, c.K, c.p)
        g.run(c.gates)
        g.close()
        b = sv.Batch(8, prec=1)
        s = b.add(c.n, c.K)
        for (q, u) in c.gates[:6]:
            b.step([(s, q, u)])
        b.close()
        torch.cuda.synchronize()

    cycle()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(8):
        cycle()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 32 << 20, (free0, free1)


@pytest.mark.parametrize("prec", [0, 1])
def test_merge_grouping_with_empty_and_lopsided_runs(sv, oracle_mod, prec):
    """Gates on qubits no earlier gate touched put every term in one run of
    the partition (the other runs empty); gates mixing fresh and used qubits
    give lopsided runs.  Checked against the oracle after every gate."""
    rng = np.random.default_rng(660 + prec)
    n = 36
    h = C.mat_h()
    gates = [((q,), h) for q in range(14)]            # 16384 terms on qubits 0..13
    gates += [((20, 30), C.haar_unitary(4, rng))]     # both fresh: one run of four
    gates += [((31, 3, 22), C.haar_unitary(8, rng))]  # two fresh, one used
    gates += [((5,), h), ((35, 34, 33, 32), C.haar_unitary(16, rng))]
    gates += [((20, 31), C.haar_unitary(4, rng)), ((0, 35), C.haar_unitary(4, rng))]
    g = sv.SparseState(n, 1 << 16, 1.0, prec=prec)
    o = oracle_mod.Oracle(n, 1 << 16, 1.0, prec=prec)
    run_both(gates, g, o)


def _random_diagonal(m, rng, kind):
    d = 1 << m
    if kind == "phase":
        return np.diag(np.exp(2j * np.pi * rng.random(d)))
    if kind == "quarter":    # entries 1, i, -1, -i: real or imaginary part exactly zero
        return np.diag((1j) ** rng.integers(0, 4, size=d)).astype(np.complex128)
    return C.mat_rz(np.pi) if m == 1 else np.diag([1.0] * (d - 1) + [-1.0]).astype(np.complex128)


@pytest.mark.parametrize("prec", [0, 1])
def test_diagonal_gates_in_place_match_oracle(sv, oracle_mod, prec):
    """Diagonal gates (phases, RZ(pi), CZ-like sign flips, entries with a zero
    real or imaginary part) update the amplitudes in place without
    regrouping; interleaved with dense gates that regroup the state, on
    states from a few terms up to several times the kernel's grid, with
    truncation after every gate."""
    rng = np.random.default_rng(880 + prec)
    for count, n, K, p in [(5, 8, 4, 1.0), (70001, 30, 50000, 0.99), (2_500_000, 36, 2_000_000, 0.9999)]:
        keys, amps = C.random_state(n, count, rng, ties=True)
        g = sv.SparseState(n, K, p, prec=prec)
        o = oracle_mod.Oracle(n, K, p, prec=prec)
        g.load(keys, amps)
        o.load(keys, amps)
        gates = []
        for step in range(6):
            m = int(rng.integers(1, min(4, n) + 1))
            qs = tuple(int(x) for x in rng.choice(n, size=m, replace=False))
            gates.append((qs, _random_diagonal(m, rng, ["phase", "quarter", "sign"][step % 3])))
            if step % 2 == 1:
                gates.append(C.random_gate(n, 1, rng, "haar"))
        run_both(gates, g, o, check_every=count < 100000)


def _random_monomial(m, rng):
    d = 1 << m
    perm = rng.permutation(d)
    u = np.zeros((d, d), dtype=np.complex128)
    phases = [1.0, -1.0, 1j, -1j, np.exp(2j * np.pi * rng.random())]
    for r in range(d):
        u[perm[r], r] = phases[int(rng.integers(0, len(phases)))]
    return u


@pytest.mark.parametrize("prec", [0, 1])
def test_monomial_gates_match_oracle(sv, oracle_mod, prec):
    """Permutations with phases on m = 1..4 qubits (X, CNOT, Toffoli, C3X and
    random ones): the regrouping sorts by the output index and one pass
    applies the entries.  Interleaved with dense and diagonal gates, with
    truncation after every gate, on states above the shared-memory size."""
    rng = np.random.default_rng(890 + prec)
    for count, n, K, p in [(5000, 20, 4000, 1.0), (300_001, 40, 250_000, 0.999)]:
        keys, amps = C.random_state(n, count, rng, ties=True)
        g = sv.SparseState(n, K, p, prec=prec)
        o = oracle_mod.Oracle(n, K, p, prec=prec)
        g.load(keys, amps)
        o.load(keys, amps)
        gates = []
        for step in range(8):
            m = 1 + step % 4
            qs = tuple(int(x) for x in rng.choice(n, size=m, replace=False))
            gates.append((qs, C.mat_mcx(m) if (step // 4) == 0 and m > 1 else _random_monomial(m, rng)))
            if step % 3 == 2:
                gates.append(C.random_gate(n, 1, rng, "haar"))
            if step % 4 == 1:
                gates.append(((int(rng.integers(0, n)),), C.mat_rz(float(rng.random()))))
        run_both(gates, g, o, check_every=count < 100000)


@pytest.mark.parametrize("prec", [0, 1])
def test_reserved_handle_allocates_nothing_and_matches(sv, oracle_mod, prec):
    """sv_reserve sizes every buffer up front: the gates and truncations that
    follow take no device memory (free memory unchanged), and the results are
    the oracle's, as on a handle that grows its buffers on demand."""
    import torch
    c = C.random_mix_circuit(30, 40, seed=17 + prec, sigma=0.05, K=1 << 14, p=0.999)
    g = sv.SparseState(c.n, c.K, c.p, prec=prec)
    g.reserve(c.K)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    o = oracle_mod.Oracle(c.n, c.K, c.p, prec=prec)
    run_both(c.gates, g, o, check_every=False)
    torch.cuda.synchronize()
    # exports allocate a staging buffer and free it again; the gates none
    assert torch.cuda.mem_get_info()[0] >= free0 - (2 << 20)
    h = sv.SparseState(c.n, c.K, c.p, prec=prec)
    h.run(c.gates)
    hk, ha = h.export()
    gk, ga = g.export()
    assert np.array_equal(hk, gk) and np.array_equal(ha, ga)
    with pytest.raises(sv.SVError):
        g.reserve(1 << 40)
