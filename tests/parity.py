"""Comparison helpers: CUDA path (through the C ABI) against the oracle."""
import functools

import numpy as np

from paper_2607_07816_b300 import circuits as C


def assert_states_equal(gpu, orc, exact=True, atol=0.0, what=""):
    """Kept key sets identical, amplitudes equal (exactly, or within atol),
    compared in canonical order (probability descending, key ascending)."""
    gk, ga = gpu.export()
    ok, oa, _ = orc.export()
    assert len(gk) == len(ok), f"{what}: term count {len(gk)} != oracle {len(ok)}"
    if not np.array_equal(gk, ok):
        sg, so = set(gk.tolist()), set(ok.tolist())
        raise AssertionError(f"{what}: key sets differ: {len(sg - so)} extra, {len(so - sg)} missing; "
                             f"first order mismatch at {int(np.argmax(gk != ok))}")
    if exact:
        bad = ~((ga.real == oa.real) & (ga.imag == oa.imag))
        assert not bad.any(), (f"{what}: {int(bad.sum())} amplitudes differ, max |d| = "
                               f"{np.max(np.abs(ga - oa)):.3e}")
    else:
        d = np.max(np.abs(ga - oa)) if len(ga) else 0.0
        assert d <= atol, f"{what}: max |d amp| {d:.3e} > {atol}"


def run_both(gates, gpu, orc, truncate=True, check_every=True, exact=True, atol=0.0):
    for t, (q, u) in enumerate(gates):
        gpu.apply_gate(q, u)
        orc.apply_gate(q, u)
        if truncate:
            kg, fg = gpu.truncate()
            ko, fo = orc.truncate()
            assert kg == ko, f"gate {t}: kept {kg} != oracle {ko}"
            assert fg == fo, f"gate {t}: retained fraction {fg!r} != oracle {fo!r}"
        if check_every:
            assert_states_equal(gpu, orc, exact=exact, atol=atol, what=f"gate {t}")
    assert_states_equal(gpu, orc, exact=exact, atol=atol, what="final")
    assert gpu.peak() == orc.peak()
    assert gpu.retained_mass() == orc.retained_mass()


@functools.lru_cache(maxsize=None)
def batched_sample(count=8, max_log2_k=11, max_gates=200):
    """The first `count` circuits of the 512-circuit batched workload (seed
    1004; circuit j depends on j alone, so the first 160 are those of the
    full list) with K <= 2^max_log2_k and at most max_gates gates (small enough
    for the oracle to finish in a few seconds)."""
    out = []
    for j, c in enumerate(C.batch_circuits(count=160)):
        if c.K <= (1 << max_log2_k) and len(c.gates) <= max_gates:
            out.append((j, c))
            if len(out) == count:
                break
    return out
