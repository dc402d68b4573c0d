"""Pins for the CPU oracle (no GPU needed).

The oracle is checked against things other than itself: a textbook dense
simulator, closed forms, invariants the paper states (Sec. I term-count
behaviour, Sec. III truncation semantics) and brute force with exact rational
arithmetic on tiny inputs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C
from tests.dense import dense_apply, dense_run, dense_zero

TWO120 = 1 << 120


def oracle_dense(o, n):
    keys, amps, _ = o.export()
    v = np.zeros(1 << n, dtype=np.complex128)
    v[keys.astype(np.int64)] = amps
    return v


# ------------------------------------------------------------ arithmetic pins
def exact_fx(p: float) -> int:
    return math.floor(Fraction(p) * TWO120)


def rn(x: Fraction) -> float:
    """Round an exact rational to the nearest double (ties to even)."""
    return float(x)


@pytest.mark.parametrize("p", [0.0, 1.0, 0.5, 2.0 ** -120, 2.0 ** -121, 3 * 2.0 ** -122,
                               1e-30, 0.1, 0.999999999, 5e-324, 2.0 ** -60 * 1.2345, 100.0])
def test_fx_matches_exact_floor(oracle_mod, p):
    assert oracle_mod.fx(p) == exact_fx(p)


def test_fx_random(oracle_mod):
    rng = np.random.default_rng(7)
    for e in rng.uniform(-130, 6, size=300):
        p = float(rng.random() * 2.0 ** e)
        assert oracle_mod.fx(p) == exact_fx(p)


def test_fx_to_double_is_correctly_rounded(oracle_mod):
    rng = np.random.default_rng(8)
    cases = [0, 1, TWO120, TWO120 - 1, (1 << 53) + 1, ((1 << 53) + 1) << 60, ((1 << 54) + 2) << 40,
             (((1 << 53) + 1) << 1) + 1]
    cases += [int(x) for x in rng.integers(0, 2 ** 63, size=50)]
    cases += [int(rng.integers(0, 2 ** 62)) << int(rng.integers(0, 64)) for _ in range(100)]
    for s in cases:
        s &= (1 << 128) - 1
        assert oracle_mod.fx_to_double(s) == rn(Fraction(s, TWO120)), s


def test_prob_definition(oracle_mod):
    # prob = RN(re^2 + RN(im^2)): one fused multiply-add over a rounded square
    rng = np.random.default_rng(9)
    for _ in range(500):
        re, im = rng.standard_normal(2) * 10.0 ** rng.uniform(-8, 0, size=2)
        want = rn(Fraction(re) ** 2 + Fraction(rn(Fraction(im) ** 2)))
        assert oracle_mod.prob(re, im) == want
    # complex64 widened components: both products exact, one rounding
    for _ in range(200):
        re, im = np.float32(rng.standard_normal()), np.float32(rng.standard_normal())
        want = rn(Fraction(float(re)) ** 2 + Fraction(float(im)) ** 2)
        assert oracle_mod.prob(float(re), float(im)) == want


# ------------------------------------------------------------ closed forms
def test_single_qubit_rule_eq3(oracle_mod):
    """Eq. (3): alpha'_0 = u00 a0 + u01 a1, alpha'_1 = u10 a0 + u11 a1."""
    o = oracle_mod.Oracle(1)
    o.load(np.array([0, 1], dtype=np.uint64), np.array([0.6, 0.8j]))
    u = np.array([[0.5 + 0.5j, 0.5 - 0.5j], [0.5 - 0.5j, 0.5 + 0.5j]])
    o.apply_gate((0,), u)
    v = oracle_dense(o, 1)
    want = u @ np.array([0.6, 0.8j])
    assert np.allclose(v, want, atol=1e-15)


def test_bell_and_ghz(oracle_mod):
    o = oracle_mod.Oracle(3)
    o.apply_gate((0,), C.mat_h())
    assert o.num_terms() == 2                     # H doubles (Sec. I)
    o.apply_gate((0, 1), C.mat_mcx(2))
    assert o.num_terms() == 2                     # CNOT permutes (Sec. I)
    keys, amps, _ = o.export()
    assert sorted(keys.tolist()) == [0, 3]
    assert np.allclose(amps, C.SQRT1_2, atol=0)
    o.apply_gate((1, 2), C.mat_mcx(2))
    keys, amps, _ = o.export()
    assert sorted(keys.tolist()) == [0, 7]
    assert np.all(amps == C.SQRT1_2)


def test_hadamard_layer_uniform(oracle_mod):
    n = 6
    o = oracle_mod.Oracle(n)
    for i in range(n):
        before = o.num_terms()
        o.apply_gate((i,), C.mat_h())
        assert o.num_terms() == 2 * before        # fresh qubit: doubling
    keys, amps, _ = o.export()
    assert len(keys) == 1 << n
    assert np.allclose(amps, 2.0 ** (-n / 2), rtol=1e-15, atol=0)


def test_x_string_and_rz_phase(oracle_mod):
    n, s = 10, 0b1011001101
    o = oracle_mod.Oracle(n)
    for (q, u) in C.x_layer(s, n):
        o.apply_gate(q, u)
    assert o.peak() == (s, 1.0)
    o.apply_gate((0,), C.mat_rz(0.7))             # bit 0 of s is 1: e^{+i 0.35}
    keys, amps, _ = o.export()
    assert keys.tolist() == [s]
    assert abs(amps[0] - np.exp(0.35j)) < 1e-16


def test_haar_two_qubit_on_fresh_qubits_quadruples(oracle_mod):
    rng = np.random.default_rng(3)
    o = oracle_mod.Oracle(8)
    o.apply_gate((2, 5), C.haar_unitary(4, rng))
    assert o.num_terms() == 4
    o.apply_gate((0, 7), C.haar_unitary(4, rng))
    assert o.num_terms() == 16


@pytest.mark.parametrize("m", [2, 3, 4])
def test_controlled_x_keeps_term_count(oracle_mod, m):
    """CNOT / Toffoli / C3X only rearrange amplitudes (Sec. I)."""
    rng = np.random.default_rng(10 + m)
    n = 9
    o = oracle_mod.Oracle(n)
    keys, amps = C.random_state(n, 200, rng)
    o.load(keys, amps)
    for _ in range(6):
        qs = tuple(int(x) for x in rng.choice(n, size=m, replace=False))
        o.apply_gate(qs, C.mat_mcx(m))
        assert o.num_terms() == 200
    o.apply_gate((3, 1), C.mat_cz())
    assert o.num_terms() == 200


# ------------------------------------------------------------ dense agreement
@pytest.mark.parametrize("seed", range(6))
def test_random_circuit_matches_dense(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 11))
    gates = []
    for _ in range(25):
        m = int(rng.integers(1, min(4, n) + 1))
        kind = rng.choice(["haar", "mcx", "h"])
        gates.append(C.random_gate(n, m, rng, str(kind)))
    o = oracle_mod.Oracle(n)
    o.run(gates, truncate=False)
    want = dense_run(n, gates)
    got = oracle_dense(o, n)
    assert np.max(np.abs(got - want)) < 1e-13
    assert abs(o.total_mass_fx() / TWO120 - 1.0) < 1e-12      # norm preserved


def test_config_mix_small_matches_dense(oracle_mod):
    c = C.random_mix_circuit(10, 40, seed=5, sigma=0.05, K=1 << 20, p=1.0)
    o = oracle_mod.Oracle(c.n)
    o.run(c.gates, truncate=False)
    assert np.max(np.abs(oracle_dense(o, c.n) - dense_run(c.n, c.gates))) < 1e-13


def test_exact_mirror_recovers_hidden_string(oracle_mod):
    c = C.exact_mirror_n12()
    o = oracle_mod.Oracle(c.n, c.K, c.p)
    o.run(c.gates)
    key, pr = o.peak()
    assert key == c.hidden
    assert pr >= 1.0 - 1e-12
    psi = dense_run(c.n, c.gates)
    assert np.max(np.abs(oracle_dense(o, c.n) - psi)) < 1e-13


def test_complex64_form_close_to_dense(oracle_mod):
    rng = np.random.default_rng(21)
    n = 9
    gates = [C.random_gate(n, int(rng.integers(1, 5)), rng, "haar") for _ in range(20)]
    o = oracle_mod.Oracle(n, prec=oracle_mod.C64)
    o.run(gates, truncate=False)
    assert np.max(np.abs(oracle_dense(o, n) - dense_run(n, gates))) < 2e-6
    _, amps, _ = o.export()
    assert np.all(amps.real.astype(np.float32).astype(np.float64) == amps.real)


# ------------------------------------------------------------ truncation
def brute_truncate(keys, amps, K, p, prec=0):
    """Sec. III rule by brute force with exact rationals: full sort, p-mass
    first, then top-k, then renormalisation."""
    probs = [rn(Fraction(float(a.real)) ** 2 + Fraction(rn(Fraction(float(a.imag)) ** 2)))
             for a in amps]
    order = sorted(range(len(keys)), key=lambda i: (-probs[i], int(keys[i])))
    fxs = [exact_fx(probs[i]) for i in order]
    SN = sum(fxs)
    N = len(keys)
    cp = N
    if p < 1.0:
        T = exact_fx(rn(Fraction(p) * Fraction(rn(Fraction(SN, TWO120)))))
        S = 0
        for c in range(1, N + 1):
            S += fxs[c - 1]
            if S >= T:
                cp = c
                break
    c = min(cp, K)
    if c == N:
        return {int(keys[i]): amps[i] for i in range(N)}, c, 1.0
    Sc = sum(fxs[:c])
    s = 1.0 / math.sqrt(rn(Fraction(Sc, TWO120)))
    out = {}
    for i in order[:c]:
        a = amps[i]
        if prec == 0:
            out[int(keys[i])] = complex(float(a.real) * s, float(a.imag) * s)
        else:
            out[int(keys[i])] = complex(float(np.float32(float(a.real) * s)),
                                        float(np.float32(float(a.imag) * s)))
    f = rn(Fraction(Sc, TWO120)) / rn(Fraction(SN, TWO120))
    return out, c, f


def _tie_state(rng, n, count):
    keys, amps = C.random_state(n, count, rng, ties=True)
    return keys, amps


@pytest.mark.parametrize("case", range(40))
def test_truncation_matches_brute_force(oracle_mod, case):
    rng = np.random.default_rng(1000 + case)
    n = int(rng.integers(3, 9))
    count = int(rng.integers(1, min(60, 1 << n) + 1))
    keys, amps = _tie_state(rng, n, count)
    K = int(rng.integers(1, count + 3))
    p = float(rng.choice([1.0, 0.5, 0.9, 0.99, 0.3, 1e-9, rng.random()]))
    o = oracle_mod.Oracle(n, K, p)
    o.load(keys, amps)
    kept, f = o.truncate()
    want, c, wf = brute_truncate(keys, amps, K, p)
    assert kept == c == len(want)
    assert f == wf
    k2, a2, _ = o.export()
    got = {int(k): a for k, a in zip(k2, a2)}
    assert got.keys() == want.keys()
    for k in got:
        assert got[k] == want[k]


def test_p_cut_lands_exactly_on_prefix_sum(oracle_mod):
    # probabilities 1/2, 1/4, 1/8, 1/8 (exact in binary); p = 3/4 must keep
    # exactly two terms (S_2 == T), p slightly above keeps three
    keys = np.array([5, 9, 2, 7], dtype=np.uint64)
    amps = np.array([0.5 + 0.5j, 0.5, 0.25 + 0.25j, -0.25 + 0.25j])
    for p, want_c in [(0.75, 2), (0.75 + 1e-12, 3), (0.5, 1), (0.875, 3), (0.99, 4)]:
        o = oracle_mod.Oracle(4, 100, p)
        o.load(keys, amps)
        kept, _ = o.truncate()
        assert kept == want_c, (p, kept)
        cut = o.last_cut()
        T = exact_fx(rn(Fraction(p) * Fraction(rn(Fraction(cut["SN"], TWO120)))))
        assert cut["Sc"] >= T


def test_equal_probabilities_break_ties_by_key(oracle_mod):
    n = 5
    o = oracle_mod.Oracle(n, 7, 1.0)
    for i in range(n):
        o.apply_gate((i,), C.mat_h())
    kept, f = o.truncate()
    keys, amps, _ = o.export()
    assert kept == 7 and sorted(keys.tolist()) == list(range(7))
    assert f == 7 / 32
    assert abs(o.total_mass_fx() / TWO120 - 1.0) < 1e-15


def test_truncation_invariants_random(oracle_mod):
    rng = np.random.default_rng(77)
    for trial in range(20):
        n = 12
        keys, amps = C.random_state(n, 500, rng, ties=bool(trial % 2))
        K = int(rng.integers(1, 600))
        p = float(rng.uniform(0.2, 1.0))
        o = oracle_mod.Oracle(n, K, p)
        o.load(keys, amps)
        keys0, _, probs0 = o.export()
        kept, f = o.truncate()
        cut = o.last_cut()
        assert kept <= K
        if kept < cut["N"]:
            # kept terms dominate the dropped ones in canonical order
            k2, _, _ = o.export()
            kept_set = set(k2.tolist())
            pk = sorted([(probs0[i], int(keys0[i])) for i in range(len(keys0))],
                        key=lambda t: (-t[0], t[1]))
            assert set(k for _, k in pk[:kept]) == kept_set
            assert abs(o.total_mass_fx() / TWO120 - 1.0) < 1e-14
            assert abs(f - cut["Sc"] / cut["SN"]) < 1e-15


def test_retained_mass_is_product(oracle_mod):
    rng = np.random.default_rng(5)
    o = oracle_mod.Oracle(10, 40, 0.95)
    fs = []
    for _ in range(8):
        o.apply_gate(tuple(int(x) for x in rng.choice(10, 2, replace=False)), C.haar_unitary(4, rng))
        fs.append(o.truncate()[1])
    want = 1.0
    for f in fs:
        want *= f
    assert o.retained_mass() == want


def test_load_rejects_bad_input(oracle_mod):
    o = oracle_mod.Oracle(4)
    with pytest.raises(ValueError):
        o.load(np.array([1, 1], dtype=np.uint64), np.array([0.6, 0.8]))
    with pytest.raises(ValueError):
        o.load(np.array([16], dtype=np.uint64), np.array([1.0]))
    with pytest.raises(ValueError):
        o.apply_gate((1, 1), np.eye(4))


# ------------------------------------------------------------ golden fixtures
def _eval_expr(s: str) -> float:
    table = {"0": 0.0, "1": 1.0, "-1": -1.0, "1/2": 0.5, "-1/2": -0.5,
             "1/sqrt(2)": 1.0 / math.sqrt(2.0), "-1/sqrt(2)": -1.0 / math.sqrt(2.0)}
    return table[s]


def _named_gate(name):
    return {"X": C.mat_x(), "H": C.mat_h(), "CNOT": C.mat_mcx(2), "TOFFOLI": C.mat_mcx(3),
            "C3X": C.mat_mcx(4), "CZ": C.mat_cz(), "RZ_PI_2": C.mat_rz(math.pi / 2)}[name]


def test_golden_closed_forms(oracle_mod):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")
    cases = json.load(open(path))["cases"]
    assert len(cases) >= 8
    for case in cases:
        o = oracle_mod.Oracle(case["n"])
        gates = [(tuple(q), _named_gate(g)) for g, q in case["gates"]]
        o.run(gates, truncate=False)
        keys, amps, _ = o.export()
        got = {int(k): a for k, a in zip(keys, amps)}
        want = {int(k): complex(_eval_expr(v[0]), _eval_expr(v[1])) for k, v in case["expect"].items()}
        assert got.keys() == want.keys(), case["name"]
        for k in want:
            assert abs(got[k] - want[k]) < 1e-15, case["name"]
        # the dense textbook simulator agrees as well
        psi = dense_run(case["n"], gates)
        for k in range(1 << case["n"]):
            assert abs(psi[k] - want.get(k, 0.0)) < 1e-15, case["name"]


# ------------------------------------------------------------ complex64 form
def rn32(x: Fraction) -> float:
    """Round an exact rational to the nearest binary32 value (ties to even,
    gradual underflow), returned as the (exactly equal) double."""
    if x == 0:
        return 0.0
    sign = -1.0 if x < 0 else 1.0
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    q = max(e - 23, -149)                  # quantum: 24-bit significand, subnormals below 2^-126
    scaled = a / Fraction(2) ** q
    n = scaled.numerator // scaled.denominator
    rem = scaled - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = Fraction(n) * Fraction(2) ** q
    assert v < Fraction(2) ** 128, "binary32 overflow"
    return sign * float(v)


def test_rn32_agrees_with_numpy_on_doubles():
    # a double rounds to binary32 once, so numpy's conversion is the reference here
    rng = np.random.default_rng(31)
    vals = list(rng.standard_normal(300) * 10.0 ** rng.uniform(-40, 30, size=300))
    vals += [1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 2.0 ** -149 * 1.5, 2.0 ** -150, 2.0 ** -127 * 3]
    for v in vals:
        assert rn32(Fraction(v)) == float(np.float32(v)), v


def _float_state(rng, n, count, ties):
    keys, amps = C.random_state(n, count, rng, ties=ties)
    return keys, amps.astype(np.complex64).astype(np.complex128)


def brute_apply_c64(keys, amps, qubits, u):
    """One gate in the complex64 form by brute force with exact rationals:
    per output, an accumulator from zero over the present inputs in
    ascending local index, each step one complex multiply-accumulate whose
    four real fused multiply-adds are evaluated exactly and rounded to
    binary32 (U rounded to binary32 first); exact zeros dropped."""
    m = len(qubits)
    d = 1 << m
    qmask = sum(1 << q for q in qubits)
    groups = {}
    for k, a in zip(keys.tolist(), amps):
        r = sum(((k >> q) & 1) << t for t, q in enumerate(qubits))
        groups.setdefault(k & ~qmask, {})[r] = a
    uf = [[(Fraction(rn32(Fraction(float(u[ro, ri].real)))), Fraction(rn32(Fraction(float(u[ro, ri].imag)))))
           for ri in range(d)] for ro in range(d)]
    out = {}
    for rest, mem in groups.items():
        for ro in range(d):
            re = im = Fraction(0)
            for ri in sorted(mem):
                ur, ui = uf[ro][ri]
                ar, ai = Fraction(float(mem[ri].real)), Fraction(float(mem[ri].imag))
                re = Fraction(rn32(ur * ar + re))
                re = Fraction(rn32(-ui * ai + re))
                im = Fraction(rn32(ur * ai + im))
                im = Fraction(rn32(ui * ar + im))
            if re == 0 and im == 0:
                continue
            key = rest | sum(((ro >> t) & 1) << q for t, q in enumerate(qubits))
            out[key] = complex(float(re), float(im))
    return out


@pytest.mark.parametrize("case", range(6))
def test_complex64_apply_matches_exact_float_brute_force(oracle_mod, case):
    rng = np.random.default_rng(3100 + case)
    n = 7
    keys, amps = _float_state(rng, n, int(rng.integers(5, 60)), ties=False)
    o = oracle_mod.Oracle(n, prec=oracle_mod.C64)
    o.load(keys, amps)
    for step in range(3):
        m = int(rng.integers(1, 5))
        q, u = C.random_gate(n, m, rng, str(rng.choice(["haar", "mcx"])))
        k0, a0, _ = o.export()
        want = brute_apply_c64(k0, a0, q, u)
        o.apply_gate(q, u)
        k1, a1, _ = o.export()
        got = {int(k): a for k, a in zip(k1, a1)}
        assert got.keys() == want.keys(), (case, step)
        for k in want:
            assert got[k] == want[k], (case, step, k)


@pytest.mark.parametrize("case", range(40))
def test_complex64_truncation_matches_brute_force(oracle_mod, case):
    """The complex64 branch of the Sec. III rule: probabilities of the widened
    components, the same exact masses, and each kept component rescaled as
    float(double(x) * s)."""
    rng = np.random.default_rng(2000 + case)
    n = int(rng.integers(3, 9))
    count = int(rng.integers(1, min(60, 1 << n) + 1))
    keys, amps = _float_state(rng, n, count, ties=True)
    K = int(rng.integers(1, count + 3))
    p = float(rng.choice([1.0, 0.5, 0.9, 0.99, 0.3, 1e-9, rng.random()]))
    o = oracle_mod.Oracle(n, K, p, prec=oracle_mod.C64)
    o.load(keys, amps)
    kept, f = o.truncate()
    want, c, wf = brute_truncate(keys, amps, K, p, prec=1)
    assert kept == c == len(want)
    assert f == wf
    k2, a2, _ = o.export()
    got = {int(k): a for k, a in zip(k2, a2)}
    assert got.keys() == want.keys()
    for k in got:
        assert got[k] == want[k]
        assert float(np.float32(got[k].real)) == got[k].real


def test_complex64_p_cut_lands_exactly_on_prefix_sum(oracle_mod):
    keys = np.array([5, 9, 2, 7, 11], dtype=np.uint64)
    amps = np.array([0.5 + 0.5j, 0.5, 0.25 + 0.25j, -0.25 + 0.25j, 0.1 + 0.2j]).astype(np.complex64)
    amps = amps.astype(np.complex128)
    for p in [0.5, 0.75, 0.875, 0.999, 1e-300]:
        for K in [1, 2, 100]:
            o = oracle_mod.Oracle(4, K, p, prec=oracle_mod.C64)
            o.load(keys, amps)
            kept, f = o.truncate()
            want, c, wf = brute_truncate(keys, amps, K, p, prec=1)
            assert (kept, f) == (c, wf), (p, K)
            k2, a2, _ = o.export()
            assert {int(k): a for k, a in zip(k2, a2)} == want


# ------------------------------------------------------------ peak tie-break
@pytest.mark.parametrize("prec", [0, 1])
def test_peak_breaks_exact_ties_by_smallest_key(oracle_mod, prec):
    """Sec. V readout in canonical order: among terms of equal largest
    probability the smallest key wins, also when smaller keys of lower
    probability come first in key order and when the tied amplitudes differ
    (a, -a, i a and conj(a) have the same probability)."""
    rng = np.random.default_rng(4000 + prec)
    for trial in range(30):
        n = 12
        count = int(rng.integers(4, 200))
        keys = rng.choice(1 << n, size=count, replace=False).astype(np.uint64)
        amps = (rng.standard_normal(count) + 1j * rng.standard_normal(count)) * 0.05
        top = complex(0.6, 0.3) if trial % 2 else complex(0.7, 0.0)
        ties = int(rng.integers(2, min(6, count) + 1))
        # the tied terms sit at the larger keys: lower-probability terms come first in key order
        order = np.argsort(keys)
        tied = order[-ties:]
        variants = [top, -top, 1j * top, top.conjugate(), -1j * top.conjugate()]
        for j, i in enumerate(tied):
            amps[i] = variants[j % len(variants)]
        if prec == 1:
            amps = amps.astype(np.complex64).astype(np.complex128)
        probs = [rn(Fraction(float(a.real)) ** 2 + Fraction(rn(Fraction(float(a.imag)) ** 2))) for a in amps]
        pmax = max(probs)
        want_key = min(int(k) for k, pr in zip(keys, probs) if pr == pmax)
        assert sum(pr == pmax for pr in probs) >= 2
        o = oracle_mod.Oracle(n, prec=prec)
        o.load(keys, amps)
        assert o.peak() == (want_key, pmax), trial
        k0, _, p0 = o.export()
        assert (int(k0[0]), p0[0]) == (want_key, pmax)
