"""bench.py's byte and FP64 model and its roofline arithmetic, on CPU, against
values worked out by hand from the per-gate definitions:

* B_method = 2 S N_in (grouping) + S (N_in + N_pre) (mat-vec) + 8 N_pre
  (select) + S (N_pre + N_kept) (compaction), the last two only when a cut
  is made; B_strict = S (N_in + N_kept); S = 8 + amplitude bytes;
* the complex128 mat-vec's FP64 work: 4 fused multiply-adds per (input,
  output) pair of a dense gate (one output per input for a monomial gate)
  plus a multiply and an fma per candidate's probability, 2 flops each;
* achieved = algorithmic bytes (or flops) per launch over the per-launch time.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats(n_in, n_pre, n_kept, selects=1):
    s1 = {"n_in": n_in, "n_pre": n_pre}
    s2 = {"n_kept": n_kept, "select_levels": 2, "selects": selects, "window_hits": 1, "window_terms": 100}
    return s1, s2


def test_dense_gate_with_a_cut_complex128():
    tot = bench.new_totals()
    s1, s2 = _stats(1000, 8000, 1000)
    bench.account_step(tot, (1, 2, 3), "dense", s1, s2, "c128", 40)
    S = 24
    assert tot["B_method"] == 2 * S * 1000 + S * 9000 + 8 * 8000 + S * 9000 == 544000
    assert tot["B_strict"] == S * 2000
    assert tot["fp64_apply"] == 2 * (4 * 1000 * 8 + 2 * 8000)
    assert tot["cuts"] == 1 and tot["gates_dense"] == 1
    # grouping (40 + 10 bits fit one word: the index is packed below the
    # key): count pass, scatter, three merge levels over 8-byte keys
    assert tot["sort_bytes"] == 1000 * (8 + 16) + 3 * 1000 * 16
    # keep flags plus the kept terms' keys and amplitudes read and written
    assert tot["compact_bytes"] == 8000 / 8 + 2 * 24 * 1000


def test_monomial_gate_without_a_cut_complex64():
    tot = bench.new_totals()
    s1, s2 = _stats(5000, 5000, 5000, selects=0)
    bench.account_step(tot, (0, 7), "mono", s1, s2, "c64", 60)
    S = 16
    assert tot["B_method"] == 2 * S * 5000 + S * 10000
    assert tot["B_strict"] == S * 10000
    assert tot["cuts"] == 0 and tot["compact_bytes"] == 0
    # complex64: FP64 only for the probabilities
    assert tot["fp64_apply"] == 2 * (2 * 5000)


def test_diagonal_gate_moves_no_sort_bytes():
    tot = bench.new_totals()
    s1, s2 = _stats(4096, 4096, 4096, selects=0)
    bench.account_step(tot, (5,), "diag", s1, s2, "c128", 60)
    assert tot["sort_bytes"] == 0 and tot["heads_bytes"] == 0
    assert tot["apply_bytes"] == 4096 * (8 + 16) * 2


def test_index_beside_the_key_when_the_packed_key_does_not_fit():
    """n + log2 N above 64 bits: the grouping keeps a 4-byte index per key."""
    a, b = bench.new_totals(), bench.new_totals()
    s1, s2 = _stats(1 << 20, 1 << 20, 1 << 20, selects=0)
    bench.account_step(a, (1,), "mono", s1, s2, "c128", 40)
    bench.account_step(b, (1,), "mono", s1, s2, "c128", 60)
    n = 1 << 20
    assert b["sort_bytes"] - a["sort_bytes"] == n * 4 + 1 * n * 8


def test_roofline_of_an_fp64_bound_mat_vec():
    tot = bench.new_totals()
    s1, s2 = _stats(1 << 20, 1 << 23, 1 << 20)
    bench.account_step(tot, (1, 2, 3), "dense", s1, s2, "c128", 60)
    # 2 ms for the one mat-vec launch, 0.5 ms for the sort
    res = {"phase_totals": tot, "phases": {"apply": (2.0, 1), "sort": (0.5, 4), "other": (9.0, 1)}}
    peaks = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0, "src": "test"}
    r = bench.roofline(res, "c128", peaks, 1.0)
    flops = tot["fp64_apply"]
    assert r["kernel"] == "apply" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / 2e-3 / 1e12, rel=1e-3)
    assert r["peak"] == pytest.approx(148 * 2 * 2 * 2000e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["hbm_frac"] == pytest.approx(tot["apply_bytes"] / 2e-3 / 6000e9, rel=1e-3)


def test_roofline_of_a_memory_bound_phase():
    tot = bench.new_totals()
    s1, s2 = _stats(1 << 20, 1 << 22, 1 << 20)
    bench.account_step(tot, (1, 2), "dense", s1, s2, "c64", 60)
    res = {"phase_totals": tot, "phases": {"apply": (0.1, 1), "sort": (0.4, 4)}}
    r = bench.roofline(res, "c64", {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0, "src": "test"}, 1.0)
    assert r["kernel"] == "sort" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["launches"] == 4
    assert r["alg_bytes_per_launch"] == round(tot["sort_bytes"] / 4)
    assert r["achieved"] == pytest.approx(tot["sort_bytes"] / 4 / 1e-4 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, rel=1e-3)


def test_attainable_time_takes_each_phase_at_its_own_roof():
    """A dense 3-qubit complex128 gate on 2^20 terms of a 60-qubit state
    (index beside the key), 2^23 candidates cut back to 2^20, one select,
    at 6000 GB/s and 1 TFLOP/s:
      mat-vec   max(2^20*28 + 2^23*32 B, 2*(2*2^23 + 4*8*2^20) flop) -> 100.663 us (FP64)
      compact   max(2^23/8 + 2*24*2^20 B, 4*2^20 flop)              ->   8.563 us (HBM)
      the rest  grouping 2^20*28 + 3*2^20*24, scan 8*2^20, window 8*2^23,
                select 16*100 bytes                                  ->  30.059 us
    """
    tot = bench.new_totals()
    s1, s2 = _stats(1 << 20, 1 << 23, 1 << 20)
    bench.account_step(tot, (1, 2, 3), "dense", s1, s2, "c128", 60)
    assert bench.attainable_ms(tot, 6000.0, 1.0) == pytest.approx(0.139286112, rel=1e-9)
