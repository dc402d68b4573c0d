"""The allocation-free peak readout agrees with the regular one.

sv_peak_noalloc serves callers that cannot allocate device memory when
they need the readout (memory owned by another runtime or pool, a fixed
device-memory budget, or a point where an allocation would stall the
device).  It works on the caller's own device arrays with a fixed scratch
array inside the library.  This file is collected last on purpose.  It
checks two calls in a row against sv_peak on the same states, through the
C ABI, with the exact comparison the other parity tests use.
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
