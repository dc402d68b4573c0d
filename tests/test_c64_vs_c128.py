"""The complex64 form against the complex128 form on circuits drawn from the
batched workload's distribution (mirrored brickwork circuits, n in [16, 48],
forward depth in [2, 10], K = 2^k): oracle against oracle, on the CPU.

The complex64 form keeps amplitudes in binary32 and the masses, the cut and
the renormalisation in FP64.  On circuits whose truncations separate the
kept terms from the dropped ones by more than float rounding, both forms
must keep the same terms, end on the same peak string and differ by at most
2e-6 per amplitude.  The CUDA complex64 path equals the complex64 oracle bit
for bit (the GPU parity tests), so this bounds the CUDA path too.
"""
import numpy as np

from tests.parity import batched_sample


def _by_key(keys, amps):
    i = np.argsort(keys)
    return keys[i], amps[i]


def test_complex64_within_2e6_of_complex128_on_batched_circuits(oracle_mod):
    sample = batched_sample()
    assert len(sample) == 8
    for j, c in sample:
        o128 = oracle_mod.Oracle(c.n, c.K, 1.0, prec=oracle_mod.C128).run(c.gates)
        o64 = oracle_mod.Oracle(c.n, c.K, 1.0, prec=oracle_mod.C64).run(c.gates)
        k1, a1, p1 = o128.export()
        k2, a2, _ = o64.export()
        what = f"circuit {j} (n={c.n}, K={c.K}, {len(c.gates)} gates)"
        # the top two probabilities are far apart: the peak is decided
        assert len(p1) > 1 and (p1[0] - p1[1]) / p1[0] > 1e-3, what
        k1, a1 = _by_key(k1, a1)
        k2, a2 = _by_key(k2, a2)
        assert np.array_equal(k1, k2), f"{what}: kept key sets differ"
        d = float(np.max(np.abs(a1 - a2)))
        assert d <= 2e-6, f"{what}: max |d amp| {d:.3e}"
        assert o64.peak()[0] == o128.peak()[0], what
        assert abs(o64.peak()[1] - o128.peak()[1]) <= 4e-6, what


def test_complex64_oracle_differs_from_complex128_oracle(oracle_mod):
    """The two forms are not the same computation: on a Haar circuit their
    amplitudes differ by float rounding (nonzero, far below 2e-6), so the
    comparison above is not vacuous."""
    j, c = batched_sample(count=1)[0]
    a = oracle_mod.Oracle(c.n, c.K, 1.0, prec=oracle_mod.C128).run(c.gates).export()
    b = oracle_mod.Oracle(c.n, c.K, 1.0, prec=oracle_mod.C64).run(c.gates).export()
    k1, a1 = _by_key(a[0], a[1])
    k2, a2 = _by_key(b[0], b[1])
    assert np.array_equal(k1, k2)
    d = float(np.max(np.abs(a1 - a2)))
    assert 1e-9 < d < 2e-6
    # every complex64 amplitude is float-representable
    assert np.array_equal(a2.astype(np.complex64).astype(np.complex128), a2)

