"""Parity at the sizes the benchmark runs: more than 2.4 M candidates.

The truncation kernels launch at most 1184 blocks of 2048-term tiles
(the window pass and the windowed compaction), so only above about 2.4 M
candidates does a block loop over several tiles: its exact mass
accumulators, its queue of above-window probabilities (the pass used after a
complex128 mat-vec), its keep-flag words and its running best kept term then
span tiles.  These cases drive those paths with 4 M candidates and compare
with the oracle exactly: kept keys, amplitudes, retained fraction and peak,
in both precisions, for top-k, p-mass then top-k, truncation straight after
a load (the pass that sums the total itself), and exact probability ties at
the cut (a Hadamard on a fresh qubit gives every output a tied twin).
The batched form gets circuits whose cut bins hold far more than the 4096
terms its select finishes in shared memory.
"""
import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C
from tests.parity import assert_states_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import sv as _sv
    _sv.load_library()
    return _sv


def _pair(sv, oracle_mod, n, K, p, prec, keys, amps):
    g = sv.SparseState(n, K, p, prec=prec)
    o = oracle_mod.Oracle(n, K, p, prec=prec)
    g.load(keys, amps)
    o.load(keys, amps)
    return g, o


def _gate_then_cut(g, o, q, u, what):
    g.apply_gate(q, u)
    o.apply_gate(q, u)
    n_pre = g.num_terms()
    assert n_pre == o.num_terms(), what
    assert g.peak() == o.peak(), what          # read from the untruncated state
    kg, fg = g.truncate()
    ko, fo = o.truncate()
    assert (kg, fg) == (ko, fo), what
    assert g.peak() == o.peak(), what          # from the compaction's per-block partials
    assert g.retained_mass() == o.retained_mass(), what
    assert_states_equal(g, o, what=what)
    return n_pre


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1.0, 0.999, 0.5])
def test_haar_gate_on_2e20_terms_then_cut(sv, oracle_mod, prec, p):
    """2^20 random terms with duplicated magnitudes, one Haar 2-qubit gate
    (about 4.2 M candidates), then the cut to K = 2^20: top-k alone, the
    p-mass select at full size followed by top-k, and a p-cut below K."""
    rng = np.random.default_rng(9100 + prec)
    n = 40
    keys, amps = C.random_state(n, 1 << 20, rng, ties=True)
    g, o = _pair(sv, oracle_mod, n, 1 << 20, p, prec, keys, amps)
    q, u = C.random_gate(n, 2, rng, "haar")
    n_pre = _gate_then_cut(g, o, q, u, f"prec={prec} p={p}")
    assert n_pre > 4 * 1000 * 1000
    # a second gate on the truncated state (sorted by the first gate's key)
    q, u = C.random_gate(n, 2, rng, "haar")
    _gate_then_cut(g, o, q, u, f"prec={prec} p={p} second gate")


@pytest.mark.parametrize("prec", [0, 1])
def test_truncation_of_a_loaded_3_5e6_term_state(sv, oracle_mod, prec):
    """A loaded state (no total mass from a mat-vec: the window pass sums it)
    of 3.5 M terms with duplicated magnitudes, cut by top-k and by p-mass."""
    rng = np.random.default_rng(9200 + prec)
    n = 44
    keys, amps = C.random_state(n, 3_500_000, rng, ties=True)
    for K, p in [(1_234_567, 1.0), (3_000_000, 0.9), (2_000_001, 0.99999)]:
        g, o = _pair(sv, oracle_mod, n, K, p, prec, keys, amps)
        assert g.peak() == o.peak()
        assert g.truncate() == o.truncate(), (K, p)
        assert g.peak() == o.peak(), (K, p)
        assert_states_equal(g, o, what=f"K={K} p={p}")


@pytest.mark.parametrize("prec", [0, 1])
def test_hadamard_ties_at_the_cut_on_4e6_candidates(sv, oracle_mod, prec):
    """H on a fresh qubit of a 2^21-term state: every output has a twin of
    exactly equal probability, so a cut at K = 2^21 + 1 (and at an odd K in
    the middle) falls between tied terms and the key decides, over 4.2 M
    candidates."""
    rng = np.random.default_rng(9300 + prec)
    n = 42
    keys, amps = C.random_state(n - 1, 1 << 21, rng, ties=True)   # qubit n-1 stays fresh
    for K in [(1 << 21) + 1, 1_500_001]:
        g, o = _pair(sv, oracle_mod, n, K, 1.0, prec, keys, amps)
        n_pre = _gate_then_cut(g, o, (n - 1,), C.mat_h(), f"K={K}")
        assert n_pre == 1 << 22


@pytest.mark.parametrize("layer", [True, False], ids=["one_launch", "kernels"])
@pytest.mark.parametrize("prec", [0, 1])
def test_batched_circuits_with_large_cut_bins(sv, oracle_mod, prec, layer):
    """Batched circuits at K = 2^16 and 2^18 on 48 qubits: their first
    select levels see cut bins of far more than 4096 terms.  Each slot
    equals its circuit run alone on the oracle, with the step as one launch
    and as separate kernels."""
    circs = [C.brickwork_circuit(48, 1, seed=77 + j, sigma=0.05, K=1 << k, p=1.0) for j, k in enumerate((16, 18))]
    b = sv.Batch(4, prec=prec)
    b.set_layer_kernel(layer)
    slots = [b.add(c.n, c.K) for c in circs]
    orcs = [oracle_mod.Oracle(c.n, c.K, 1.0, prec=prec) for c in circs]
    length = max(len(c.gates) for c in circs)
    for t in range(length):
        gates = []
        for s, c, o in zip(slots, circs, orcs):
            if t < len(c.gates):
                q, u = c.gates[t]
                gates.append((s, q, u))
                o.apply_gate(q, u)
                o.truncate()
        b.step(gates)
    for s, c, o in zip(slots, circs, orcs):
        gk, ga = b.export(s)
        ok, oa, _ = o.export()
        assert len(ok) == c.K
        g = {int(k): complex(a) for k, a in zip(gk, ga)}
        w = {int(k): complex(a) for k, a in zip(ok, oa)}
        assert g.keys() == w.keys(), f"K={c.K}"
        assert all(g[k] == w[k] for k in w), f"K={c.K}"
        assert b.peak(s) == o.peak()
        assert b.retained_mass(s) == o.retained_mass()
    b.close()
