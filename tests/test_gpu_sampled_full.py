"""Sampled parity at the benchmark's full size, in the benchmark's launch
configuration: the n = 60 random-mix circuit with K = 2^26 and p = 0.9999,
buffers reserved for K-term states, run from |0> until the state holds K
terms, then five more gates, then two checked gates: the first two gates
that the benchmark times, on the full 2^26-term state (a monomial gate on 4
qubits, then a Haar U(8) gate on 3 qubits whose candidates are cut back to
2^26 terms).

The oracle cannot run a 2^26-term state, but it can compute any one partner
group (Eq. 3) from the exported input terms.  For every gate checked:

* groups of sampled input terms and of sampled output terms are recomputed
  by the oracle (same arithmetic, so the same bits as the device before the
  cut);
* a candidate is kept exactly when it precedes the cut term (the last kept
  term, itself recomputed by the oracle) in the canonical order (probability
  descending, key ascending, probabilities by the oracle's formula), Sec. III;
* kept amplitudes equal the candidate times s = 1 / sqrt(S_c) bit for bit
  (complex64: the product rounded to float), and no output term lies
  outside its group's candidates;
* the kept count is K, or fewer only when the p-mass cut came first; the
  retained product is multiplied by S_c / S_N; the renormalised state has
  unit norm; the readout is the canonical first term (Sec. V).
"""
import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C

pytestmark = pytest.mark.gpu

N_QUBITS, K, P = 60, 1 << 26, 0.9999
SAMPLES = 3000
CUT_WINDOW = 256


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import sv as _sv
    _sv.load_library()
    return _sv


def _by_key(keys, amps):
    """Keys ascending with their amplitudes (sorted on the device: 2^26 keys)."""
    import torch
    if torch.cuda.is_available():
        t = torch.from_numpy(keys.view(np.int64)).cuda()
        sk, perm = torch.sort(t)
        perm = perm.cpu().numpy()
        return sk.cpu().numpy().view(np.uint64), amps[perm]
    perm = np.argsort(keys, kind="stable")
    return keys[perm], amps[perm]


def _lookup(sorted_keys, q):
    pos = np.searchsorted(sorted_keys, q)
    pos = np.minimum(pos, len(sorted_keys) - 1)
    return pos, sorted_keys[pos] == q


def _members(bases, qubits):
    """Keys of every local index r of each group base (bit t of r = qubit q[t])."""
    m = len(qubits)
    r = np.arange(1 << m, dtype=np.uint64)
    dep = np.zeros(1 << m, dtype=np.uint64)
    for t, qb in enumerate(qubits):
        dep |= ((r >> np.uint64(t)) & np.uint64(1)) << np.uint64(qb)
    return bases[:, None] | dep[None, :]


def _group_outputs(oracle_mod, prec, qubits, u, base, kin, ain):
    """The oracle's candidates of one partner group: its present input
    members loaded alone, the gate applied, nothing truncated."""
    keys = _members(np.array([base], dtype=np.uint64), qubits)[0]
    pos, found = _lookup(kin, keys)
    o = oracle_mod.Oracle(N_QUBITS, 1 << 62, 1.0, prec=prec)
    o.load(keys[found], ain[pos[found]])
    o.apply_gate(qubits, u)
    k, a, _ = o.export()
    return k, a


def _check_gate(oracle_mod, prec, qubits, u, before, after, st_out, rng):
    kin, ain = before
    kout_c, aout_c = after          # canonical order
    n_pre, kept, f, S_N, S_c, F0, F1, peak = st_out
    assert len(kout_c) == kept
    # the count: K, or fewer only when the p-mass cut comes first
    assert kept <= K
    if kept < min(K, n_pre):
        assert S_c >= P * S_N * (1 - 1e-12)
    cut = kept < n_pre
    s = 1.0 / np.sqrt(S_c) if cut else 1.0
    if cut:
        assert f == S_c / S_N
    assert F1 == F0 * f
    if cut:
        norm = float(np.sum(np.abs(aout_c) ** 2))
        assert abs(norm - 1.0) < (1e-9 if prec == 0 else 1e-6), norm
    # readout: the canonical first term
    assert peak[0] == int(kout_c[0])
    assert peak[1] == oracle_mod.prob(aout_c[0].real, aout_c[0].imag)
    kout, aout = _by_key(kout_c, aout_c)

    mask = np.uint64(0)
    for qb in qubits:
        mask |= np.uint64(1) << np.uint64(qb)
    # the cut term: the last kept term in the canonical order of the values
    # before the rescale.  The rescale (and for complex64 its rounding to
    # float) can reorder nearly equal neighbours, so the last CUT_WINDOW
    # terms of the exported order are recomputed from their groups.
    p_cut, kc = None, None
    for key in kout_c[-CUT_WINDOW:]:
        gk, ga = _group_outputs(oracle_mod, prec, qubits, u, key & ~mask, kin, ain)
        j = int(np.nonzero(gk == key)[0][0])
        pr = oracle_mod.prob(ga[j].real, ga[j].imag)
        if p_cut is None or pr < p_cut or (pr == p_cut and int(key) > kc):
            p_cut, kc = pr, int(key)

    bases = np.unique(np.concatenate([
        kin[rng.integers(0, len(kin), SAMPLES)] & ~mask,
        kout[rng.integers(0, len(kout), SAMPLES)] & ~mask]))
    n_kept = n_dropped = 0
    for b in bases:
        gk, ga = _group_outputs(oracle_mod, prec, qubits, u, b, kin, ain)
        pos, found = _lookup(kout, gk)
        for key, a, i, hit in zip(gk, ga, pos, found):
            pr = oracle_mod.prob(a.real, a.imag)
            precedes = pr > p_cut or (pr == p_cut and int(key) <= kc)
            assert hit == precedes, (int(key), pr, p_cut, bool(hit))
            if hit:
                want = complex(a.real * s, a.imag * s)
                if prec == 1:
                    want = complex(np.float32(a.real * s), np.float32(a.imag * s))
                assert aout[i] == want, (int(key), aout[i], want)
                n_kept += 1
            else:
                n_dropped += 1
        # every output term of this group is one of its candidates
        outs = _members(np.array([b], dtype=np.uint64), qubits)[0]
        _, present = _lookup(kout, outs)
        assert set(outs[present].tolist()) <= set(gk.tolist())
    return n_kept, n_dropped, len(bases)


@pytest.mark.parametrize("prec", [0, 1])
def test_sampled_parity_on_the_full_size_workload(sv, oracle_mod, prec):
    circ = C.mix_n60(K=K, p=P)
    st = sv.SparseState(N_QUBITS, K, P, prec=prec)
    st.reserve(K)
    gi = 0
    while gi < len(circ.gates) and st.num_terms() < 0.99 * K:
        st.apply_gate(*circ.gates[gi])
        st.truncate()
        gi += 1
    for _ in range(5):
        st.apply_gate(*circ.gates[gi])
        st.truncate()
        gi += 1
    rng = np.random.default_rng(4401 + prec)
    before = _by_key(*st.export())
    seen = []
    for _ in range(2):
        q, u = circ.gates[gi]
        gi += 1
        F0 = st.retained_mass()
        st.apply_gate(q, u)
        n_pre = st.stats()["n_pre"]
        kept, f = st.truncate()
        stats = st.stats()
        after = st.export()
        out = (n_pre, kept, f, stats["total_mass"], stats["kept_mass"], F0, st.retained_mass(), st.peak())
        n_kept, n_dropped, groups = _check_gate(oracle_mod, prec, q, u, before, after, out, rng)
        assert groups > SAMPLES and n_kept > 0
        seen.append((len(q), n_pre, kept, n_dropped))
        before = _by_key(*after)
    print(f"checked gates {gi - 2}, {gi - 1}: (m, candidates, kept, sampled candidates dropped) = {seen}")
    # the checked gates work on full states, and at least one of them cuts
    # candidates that the sample then sees dropped
    assert all(kept > 0.99 * K for _, _, kept, _ in seen), seen
    assert any(n_pre > kept and d > 0 for _, n_pre, kept, d in seen), seen
    st.close()
