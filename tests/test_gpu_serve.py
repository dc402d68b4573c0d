"""Serving form on the GPU: each circuit's result is the same alone and in the
mix of a continuous-batching run (requests arriving while others are
resident, admission held back by the byte budget), and matches the oracle:
exactly in the batch's own precision, within 2e-6 per amplitude of the
complex128 oracle for complex64, with identical peaks."""
import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import serve as _serve
    from paper_2607_07816_b300 import sv as _sv
    _sv.load_library()
    return _serve


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = int(rng.integers(10, 27))
        depth = int(rng.integers(1, 4))
        K = 1 << int(rng.integers(5, 12))
        out.append(C.brickwork_circuit(n, depth, seed=int(rng.integers(1 << 30)), sigma=0.05, K=K, p=1.0))
    return out


def _as_dict(keys, amps):
    return {int(k): complex(a) for k, a in zip(keys, amps)}


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("one_launch", [True, False], ids=["one_launch", "kernels"])
def test_alone_vs_mix(serve, oracle_mod, prec, one_launch):
    circs = _requests(14, 900 + prec)
    # arrivals in steps: later requests arrive while earlier ones are resident
    arrivals = [0, 0, 1, 3, 4, 4, 7, 9, 12, 12, 15, 20, 22, 30]
    budget = 3 * max(serve.footprint(c) for c in circs)
    srv = serve.Server(budget, max_slots=6, prec=prec, one_launch=one_launch)
    mix = srv.run(circs, arrivals=arrivals, clock=lambda: srv.steps, export=True)
    assert srv.peak_bytes <= budget and srv.peak_resident >= 2
    srv.close()
    # the same stream with pipelined readouts (no export): the same results
    srv = serve.Server(budget, max_slots=6, prec=prec, one_launch=one_launch)
    piped = srv.run(circs, arrivals=arrivals, clock=lambda: srv.steps)
    srv.close()
    for m, q in zip(mix, piped):
        assert (m.peak_key, m.peak_prob, m.retained_mass) == (q.peak_key, q.peak_prob, q.retained_mass)
    for j, c in enumerate(circs):
        one = serve.Server(1 << 40, max_slots=1, prec=prec, one_launch=one_launch)
        alone = one.run([c], export=True)[0]
        one.close()
        m = mix[j]
        assert (m.peak_key, m.peak_prob, m.retained_mass) == (alone.peak_key, alone.peak_prob, alone.retained_mass)
        assert _as_dict(m.keys, m.amps) == _as_dict(alone.keys, alone.amps), f"request {j}"
        # same precision oracle: exact
        o = oracle_mod.Oracle(c.n, c.K, 1.0, prec=prec)
        o.run(c.gates)
        ok, oa, _ = o.export()
        assert _as_dict(ok, oa) == _as_dict(m.keys, m.amps), f"request {j} vs oracle"
        assert o.peak() == (m.peak_key, m.peak_prob)
        if prec == 1:
            o128 = oracle_mod.Oracle(c.n, c.K, 1.0, prec=0)
            o128.run(c.gates)
            assert o128.peak()[0] == m.peak_key
            k128, a128, _ = o128.export()
            d128 = _as_dict(k128, a128)
            common = [k for k in _as_dict(m.keys, m.amps) if k in d128]
            assert len(common) >= 0.9 * len(d128)
            gm = _as_dict(m.keys, m.amps)
            assert max(abs(gm[k] - d128[k]) for k in common) <= 2e-6


def test_serving_stream_completes_with_large_request(serve):
    """A short Poisson stream from the serving distribution at reduced sizes,
    one large n=56 request among them: every result equals the single-state
    path's result for that circuit in the same precision."""
    from paper_2607_07816_b300 import sv
    circs = [C.serving_request(j, seed=77, large_frac=0.0, k_range=(6, 10), depth_range=(1, 3))
             for j in range(30)]
    circs[5] = C.brickwork_circuit(56, 2, seed=5, sigma=0.05, K=1 << 12, p=1.0)
    arrivals = serve.poisson_arrivals(len(circs), 200.0, 3)
    srv = serve.Server(160 << 30, n_max=56, prec=1)
    assert srv.max_slots == 255
    res = srv.run(circs, arrivals=arrivals)
    srv.close()
    for r, c in zip(res, circs):
        g = sv.SparseState(c.n, c.K, 1.0, prec=1)
        g.run(c.gates)
        assert (r.peak_key, r.peak_prob) == g.peak()
        assert r.retained_mass == g.retained_mass()
        g.close()
        assert r.finished >= r.admitted >= r.arrival
    p50, p99 = serve.percentiles(res)
    assert 0 < p50 <= p99


def test_solo_lane_results_equal_single_state_path(serve):
    """Requests at or above solo_min_terms run on single-state handles of
    their own beside the batch: each result equals the single-state path's
    result for that circuit in the same precision, bit for bit."""
    from paper_2607_07816_b300 import sv
    circs = [C.serving_request(j, seed=91, large_frac=0.0, k_range=(6, 12), depth_range=(1, 3))
             for j in range(24)]
    circs[3] = C.brickwork_circuit(56, 2, seed=6, sigma=0.05, K=1 << 12, p=1.0)
    arrivals = serve.poisson_arrivals(len(circs), 300.0, 4)
    srv = serve.Server(160 << 30, n_max=56, prec=1, solo_min_terms=1 << 11)
    res = srv.run(circs, arrivals=arrivals, export=True)
    srv.close()
    assert srv.solo_served == sum(1 for c in circs if c.K >= 1 << 11) >= 2
    for r, c in zip(res, circs):
        g = sv.SparseState(c.n, c.K, 1.0, prec=1)
        g.run(c.gates)
        assert (r.peak_key, r.peak_prob) == g.peak()
        assert r.retained_mass == g.retained_mass()
        gk, ga = g.export()
        assert _as_dict(r.keys, r.amps) == _as_dict(gk, ga)
        g.close()
