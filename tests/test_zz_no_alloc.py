"""The allocation-free peak readout agrees with the regular one.

sv_peak_noalloc serves callers that cannot allocate device memory when
they need the readout (memory owned by another runtime or pool, a fixed
device-memory budget, or a point where an allocation would stall the
device).  It works on the caller's own device arrays with a fixed scratch
array inside the library.  This file is collected last on purpose.  It
checks two calls in a row against sv_peak on the same states, through the
C ABI, with the exact comparison the other parity tests use, and states
large enough for several blocks (the cross-block reduction through the
scratch array) with exact ties between blocks against the oracle.
"""
import ctypes

import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import sv
    sv.load_library()
    return sv, torch


def _device_copy(torch, keys, amps, prec):
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    if prec == 0:
        da = torch.from_numpy(amps.astype(np.complex128).view(np.float64).copy()).cuda()
    else:
        da = torch.from_numpy(amps.astype(np.complex64).view(np.float32).copy()).cuda()
    return dk, da


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_peak_matches_sv_peak_on_two_calls(env, prec):
    sv, torch = env
    rng = np.random.default_rng(2024 + prec)
    stream = torch.cuda.current_stream().cuda_stream
    st = sv.SparseState(22, 50000, 1.0, prec=prec)
    for call in range(2):
        # a different state for each call: more gates before the second one
        for _ in range(6 + 3 * call):
            m = int(rng.integers(1, 4))
            st.apply_gate(*C.random_gate(22, m, rng, "haar"))
            st.truncate()
        want = st.peak()
        keys, amps = st.export()
        dk, da = _device_copy(torch, keys, amps, prec)
        torch.cuda.synchronize()
        got = sv.sv_peak_noalloc(prec, dk.data_ptr(), da.data_ptr(), len(keys), stream)
        assert got == want, (call, got, want)


def _tied_state(rng, count, tie_pos, prec):
    """count random terms; the largest probability is shared exactly by the
    terms at array positions tie_pos (amplitudes a, -a, conj(a), i a, ...),
    and the smallest of their keys sits at the last of those positions."""
    keys = np.unique(rng.integers(0, 1 << 40, size=count + count // 8, dtype=np.uint64))[:count]
    rng.shuffle(keys)
    amps = (rng.standard_normal(count) + 1j * rng.standard_normal(count)) * 1e-3
    top = complex(0.375, -0.25)
    variants = [top, -top, top.conjugate(), 1j * top]
    tied_keys = np.sort(keys[tie_pos])[::-1]          # descending: the smallest key goes last
    keys[tie_pos] = tied_keys
    for j, i in enumerate(tie_pos):
        amps[i] = variants[j % len(variants)]
    if prec == 1:
        amps = amps.astype(np.complex64)
    return keys, amps.astype(np.complex128), int(tied_keys[-1])


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_peak_across_blocks_with_ties_matches_oracle(env, oracle_mod, prec):
    """States of 196608 to 300000 terms span 3 to 5 blocks of 65536 terms,
    so the per-block partials go through the shared scratch array and the
    last block's reduction.  The largest probability is tied between terms
    in different blocks with the smallest key in the last of them.  Two
    calls in a row on different states; each result equals the oracle's
    peak and sv_peak's on the same terms."""
    sv, torch = env
    rng = np.random.default_rng(4242 + prec)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(300_000, [70_000, 140_001, 299_999]), (3 * 65536 + 1, [5, 65536, 3 * 65536]),
             (3 * 65536, [65535, 131072, 196607])]
    for call, (count, tie_pos) in enumerate(cases):
        keys, amps, want_key = _tied_state(rng, count, tie_pos, prec)
        o = oracle_mod.Oracle(41, prec=prec)
        o.load(keys, amps)
        want = o.peak()
        assert want[0] == want_key
        st = sv.SparseState(41, prec=prec)
        st.load(keys, amps)
        assert st.peak() == want
        dk, da = _device_copy(torch, keys, amps, prec)
        torch.cuda.synchronize()
        got = sv.sv_peak_noalloc(prec, dk.data_ptr(), da.data_ptr(), count, stream)
        assert got == want, (call, got, want)


def test_noalloc_peak_rejects_sizes_beyond_its_scratch(env):
    sv, torch = env
    lib = sv.load_library()
    dk = torch.zeros(4, dtype=torch.int64, device="cuda")
    da = torch.zeros(8, dtype=torch.float64, device="cuda")
    k, p = ctypes.c_uint64(), ctypes.c_double()
    for n in (0, (1 << 28) + 1):
        rc = lib.sv_peak_noalloc(0, ctypes.c_void_p(dk.data_ptr()), ctypes.c_void_p(da.data_ptr()),
                                 ctypes.c_uint64(n), None, ctypes.byref(k), ctypes.byref(p))
        assert rc == sv.SV_E_ARG
