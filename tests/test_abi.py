"""The C ABI library builds, loads and exports every declared symbol (no GPU
needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(svb?_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_07816_b300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["sv_create", "sv_create_ex", "sv_destroy", "sv_apply_gate", "sv_truncate",
                 "sv_peak", "sv_probs", "sv_num_terms", "sv_retained_mass", "sv_export", "sv_load",
                 "sv_last_error", "svb_create", "svb_add", "svb_step", "svb_peak", "svb_peak_async",
                 "svb_peak_wait", "svb_set_layer_kernel"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2607_07816_b300 import sv
    for name in declared_symbols():
        assert name in sv.EXPORTED, name
        assert callable(getattr(sv, name)), name


def test_null_arguments_rejected_without_gpu(lib):
    # argument validation happens on the host before any CUDA call
    lib.sv_create_ex.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.sv_create_ex(0, ctypes.c_uint64(1), ctypes.c_double(1.0), 0, None, None,
                            ctypes.byref(out)) == -1
    assert lib.sv_create_ex(65, ctypes.c_uint64(1), ctypes.c_double(1.0), 0, None, None,
                            ctypes.byref(out)) == -1
    assert lib.sv_create_ex(10, ctypes.c_uint64(0), ctypes.c_double(1.0), 0, None, None,
                            ctypes.byref(out)) == -1
    assert lib.sv_create_ex(10, ctypes.c_uint64(5), ctypes.c_double(1.5), 0, None, None,
                            ctypes.byref(out)) == -1
    assert lib.sv_create_ex(10, ctypes.c_uint64(5), ctypes.c_double(0.5), 7, None, None,
                            ctypes.byref(out)) == -1
    lib.sv_destroy.restype = ctypes.c_int
    assert lib.sv_destroy(None) == 0
    lib.sv_last_error.restype = ctypes.c_char_p
    assert lib.sv_last_error(None) == b"null handle"
