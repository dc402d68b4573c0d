"""Thin Python binding of libsv.so (C ABI in include/sv.h).

Argument marshalling only: every step of gate application, truncation and
readout runs in the library's CUDA kernels.  The module-level functions carry
the C names (``sv_create``, ``sv_apply_gate``, ...); ``SparseState`` wraps a
handle for convenience.  There is no fallback: if the library cannot be
loaded, or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

SV_OK, SV_E_ARG, SV_E_NOMEM, SV_E_CUDA, SV_E_NOT_UNITARY, SV_E_TIMEOUT, SV_E_STATE = 0, -1, -2, -3, -4, -5, -6
SV_C128, SV_C64 = 0, 1
_STATUS = {0: "SV_OK", -1: "SV_E_ARG", -2: "SV_E_NOMEM", -3: "SV_E_CUDA", -4: "SV_E_NOT_UNITARY",
           -5: "SV_E_TIMEOUT", -6: "SV_E_STATE"}

EXPORTED = ["sv_create", "sv_create_ex", "sv_destroy", "sv_apply_gate", "sv_truncate", "sv_peak",
            "sv_peak_async", "sv_peak_wait",
            "sv_probs", "sv_num_terms", "sv_retained_mass", "sv_export", "sv_load", "sv_last_error",
            "sv_last_stats", "sv_set_timing", "sv_phase_times", "sv_launch_count", "sv_transfer_bytes", "sv_peak_noalloc",
            "svb_create", "svb_destroy", "svb_add", "svb_remove", "svb_step", "svb_num_terms",
            "svb_retained_mass", "svb_peak", "svb_export", "svb_last_error", "svb_set_autotune",
            "svb_autotune_stats", "svb_set_graphs", "svb_graph_stats", "svb_set_layer_kernel", "svb_layer_phase_times", "svb_peak_async", "svb_peak_wait",
            "sv_selftest", "sv_set_apply_variant",
            "sv_probe_fp64", "sv_select_histogram", "sv_cut", "sv_reserve"]
PHASES = ["keys", "sort", "heads", "apply", "select", "compact", "peak", "other", "window", "local"]


class SVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class sv_allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)),
                ("ctx", ctypes.c_void_p)]


class svb_gate(ctypes.Structure):
    _fields_ = [("slot", ctypes.c_int), ("m", ctypes.c_int), ("qubits", ctypes.c_int * 4),
                ("U", ctypes.POINTER(ctypes.c_double))]


class sv_stats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_uint64), ("n_pre", ctypes.c_uint64), ("n_kept", ctypes.c_uint64),
                ("sort_passes", ctypes.c_uint32), ("select_levels", ctypes.c_uint32),
                ("total_mass", ctypes.c_double), ("kept_mass", ctypes.c_double),
                ("window_hits", ctypes.c_uint32), ("selects", ctypes.c_uint32), ("window_terms", ctypes.c_uint64),
                ("local_gates", ctypes.c_uint64), ("global_gates", ctypes.c_uint64),
                ("local_fallbacks", ctypes.c_uint64), ("diag_gates", ctypes.c_uint64),
                ("mono_gates", ctypes.c_uint64)]


_lib = None


def lib_path() -> str:
    """The library loaded: $SV_LIBRARY when set (another build of the same
    sources, e.g. for A/B timing), else libsv.so in the package directory."""
    return os.environ.get("SV_LIBRARY") or _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsv.so from the package directory (building it when absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if path != _build.LIB and not os.path.exists(path):
        raise OSError(f"SV_LIBRARY={path} does not exist")
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"libsv.so not found at {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    P, u64, i32, dbl, vp = ctypes.POINTER, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.sv_create.restype = i32
    lib.sv_create.argtypes = [i32, u64, dbl, P(vp)]
    lib.sv_create_ex.restype = i32
    lib.sv_create_ex.argtypes = [i32, u64, dbl, i32, vp, P(sv_allocator), P(vp)]
    lib.sv_destroy.restype = i32
    lib.sv_destroy.argtypes = [vp]
    lib.sv_apply_gate.restype = i32
    lib.sv_apply_gate.argtypes = [vp, i32, P(ctypes.c_int), P(dbl)]
    lib.sv_truncate.restype = i32
    lib.sv_truncate.argtypes = [vp, P(u64), P(dbl)]
    lib.sv_peak.restype = i32
    lib.sv_peak.argtypes = [vp, P(u64), P(dbl)]
    lib.sv_peak_async.restype = i32
    lib.sv_peak_async.argtypes = [vp, P(u64)]
    lib.sv_peak_wait.restype = i32
    lib.sv_peak_wait.argtypes = [vp, u64, P(u64), P(dbl)]
    lib.sv_probs.restype = i32
    lib.sv_probs.argtypes = [vp, vp, vp, u64, P(u64)]
    lib.sv_num_terms.restype = i32
    lib.sv_num_terms.argtypes = [vp, P(u64)]
    lib.sv_retained_mass.restype = i32
    lib.sv_retained_mass.argtypes = [vp, P(dbl)]
    lib.sv_export.restype = i32
    lib.sv_export.argtypes = [vp, vp, vp, u64, P(u64)]
    lib.sv_load.restype = i32
    lib.sv_load.argtypes = [vp, vp, vp, u64]
    lib.sv_last_error.restype = ctypes.c_char_p
    lib.sv_last_error.argtypes = [vp]
    lib.sv_last_stats.restype = i32
    lib.sv_last_stats.argtypes = [vp, P(sv_stats)]
    lib.sv_set_timing.restype = i32
    lib.sv_set_timing.argtypes = [vp, i32]
    lib.sv_phase_times.restype = i32
    lib.sv_phase_times.argtypes = [vp, P(dbl), P(u64)]
    lib.sv_launch_count.restype = u64
    lib.sv_launch_count.argtypes = []
    lib.svb_create.restype = i32
    lib.svb_create.argtypes = [i32, i32, vp, P(sv_allocator), P(vp)]
    lib.svb_destroy.restype = i32
    lib.svb_destroy.argtypes = [vp]
    lib.svb_add.restype = i32
    lib.svb_add.argtypes = [vp, i32, u64, dbl, P(ctypes.c_int)]
    lib.svb_remove.restype = i32
    lib.svb_remove.argtypes = [vp, i32]
    lib.svb_step.restype = i32
    lib.svb_step.argtypes = [vp, vp, i32]
    lib.svb_num_terms.restype = i32
    lib.svb_num_terms.argtypes = [vp, i32, P(u64)]
    lib.svb_retained_mass.restype = i32
    lib.svb_retained_mass.argtypes = [vp, i32, P(dbl)]
    lib.svb_peak.restype = i32
    lib.svb_peak.argtypes = [vp, i32, P(u64), P(dbl)]
    lib.svb_export.restype = i32
    lib.svb_export.argtypes = [vp, i32, vp, vp, u64, P(u64)]
    lib.svb_last_error.restype = ctypes.c_char_p
    lib.svb_last_error.argtypes = [vp]
    lib.svb_set_autotune.restype = i32
    lib.svb_set_autotune.argtypes = [vp, i32]
    lib.svb_autotune_stats.restype = i32
    lib.svb_autotune_stats.argtypes = [vp, P(u64), P(u64), P(u64)]
    lib.svb_set_graphs.restype = i32
    lib.svb_set_graphs.argtypes = [vp, i32]
    lib.svb_set_layer_kernel.restype = i32
    lib.svb_set_layer_kernel.argtypes = [vp, i32]
    lib.svb_layer_phase_times.restype = i32
    lib.svb_layer_phase_times.argtypes = [vp, P(dbl), i32, P(i32)]
    lib.svb_peak_async.restype = i32
    lib.svb_peak_async.argtypes = [vp, i32, P(u64)]
    lib.svb_peak_wait.restype = i32
    lib.svb_peak_wait.argtypes = [vp, u64, P(u64), P(dbl), P(dbl)]
    lib.svb_graph_stats.restype = i32
    lib.svb_graph_stats.argtypes = [vp, P(u64), P(u64)]
    lib.sv_peak_noalloc.restype = i32
    lib.sv_peak_noalloc.argtypes = [i32, vp, vp, u64, vp, P(u64), P(dbl)]
    lib.sv_set_apply_variant.restype = i32
    lib.sv_set_apply_variant.argtypes = [vp, i32]
    lib.sv_selftest.restype = i32
    lib.sv_selftest.argtypes = [i32, u64, u64, P(u64), P(u64)]
    lib.sv_probe_fp64.restype = i32
    lib.sv_probe_fp64.argtypes = [u64, i32, P(dbl), P(dbl)]
    lib.sv_select_histogram.restype = i32
    lib.sv_select_histogram.argtypes = [vp, u64, u64, i32, vp, vp]
    lib.sv_reserve.restype = i32
    lib.sv_reserve.argtypes = [vp, u64]
    lib.sv_cut.restype = i32
    lib.sv_cut.argtypes = [vp, u64, u64, u64, u64, u64, u64, P(u64)]
    lib.sv_transfer_bytes.restype = None
    lib.sv_transfer_bytes.argtypes = [P(u64), P(u64)]
    _lib = lib
    return lib


def _check(h, rc: int) -> None:
    if rc != SV_OK:
        msg = _lib.sv_last_error(h).decode() if h else ""
        raise SVError(rc, msg)


def _u_buffer(u) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.complex128))
    return np.ascontiguousarray(u.view(np.float64).reshape(-1))


# ------------------------------------------------ C-named thin wrappers
def sv_create(n: int, K: int, p: float) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(None, lib.sv_create(n, ctypes.c_uint64(K), p, ctypes.byref(h)))
    return h.value


def sv_create_ex(n: int, K: int, p: float, prec: int = SV_C128, stream: int = 0) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(None, lib.sv_create_ex(n, ctypes.c_uint64(K), p, prec, ctypes.c_void_p(stream), None,
                                  ctypes.byref(h)))
    return h.value


def sv_destroy(h: int) -> None:
    _check(h, load_library().sv_destroy(ctypes.c_void_p(h)))


def sv_apply_gate(h: int, qubits: Sequence[int], u) -> None:
    lib = load_library()
    m = len(qubits)
    q = (ctypes.c_int * m)(*[int(x) for x in qubits])
    ub = _u_buffer(u)
    _check(h, lib.sv_apply_gate(ctypes.c_void_p(h), m, q, ub.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def sv_truncate(h: int):
    kept, f = ctypes.c_uint64(), ctypes.c_double()
    _check(h, load_library().sv_truncate(ctypes.c_void_p(h), ctypes.byref(kept), ctypes.byref(f)))
    return kept.value, f.value


def sv_peak(h: int):
    k, p = ctypes.c_uint64(), ctypes.c_double()
    _check(h, load_library().sv_peak(ctypes.c_void_p(h), ctypes.byref(k), ctypes.byref(p)))
    return k.value, p.value


def sv_peak_async(h: int) -> int:
    t = ctypes.c_uint64()
    _check(h, load_library().sv_peak_async(ctypes.c_void_p(h), ctypes.byref(t)))
    return t.value


def sv_peak_wait(h: int, ticket: int):
    k, p = ctypes.c_uint64(), ctypes.c_double()
    _check(h, load_library().sv_peak_wait(ctypes.c_void_p(h), ctypes.c_uint64(ticket), ctypes.byref(k),
                                          ctypes.byref(p)))
    return k.value, p.value


def sv_num_terms(h: int) -> int:
    n = ctypes.c_uint64()
    _check(h, load_library().sv_num_terms(ctypes.c_void_p(h), ctypes.byref(n)))
    return n.value


def sv_retained_mass(h: int) -> float:
    f = ctypes.c_double()
    _check(h, load_library().sv_retained_mass(ctypes.c_void_p(h), ctypes.byref(f)))
    return f.value


def sv_probs(h: int, cap: Optional[int] = None):
    n = sv_num_terms(h) if cap is None else cap
    keys = np.zeros(n, dtype=np.uint64)
    probs = np.zeros(n, dtype=np.float64)
    cnt = ctypes.c_uint64()
    _check(h, load_library().sv_probs(ctypes.c_void_p(h), keys.ctypes.data, probs.ctypes.data,
                                      ctypes.c_uint64(n), ctypes.byref(cnt)))
    w = min(n, cnt.value)
    return keys[:w], probs[:w]


def sv_export(h: int):
    n = sv_num_terms(h)
    keys = np.zeros(n, dtype=np.uint64)
    amps = np.zeros(2 * n, dtype=np.float64)
    cnt = ctypes.c_uint64()
    _check(h, load_library().sv_export(ctypes.c_void_p(h), keys.ctypes.data, amps.ctypes.data,
                                       ctypes.c_uint64(n), ctypes.byref(cnt)))
    return keys, amps.view(np.complex128)


def sv_load(h: int, keys, amps) -> None:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    a = np.ascontiguousarray(np.asarray(amps, dtype=np.complex128)).view(np.float64)
    _check(h, load_library().sv_load(ctypes.c_void_p(h), keys.ctypes.data, a.ctypes.data,
                                     ctypes.c_uint64(len(keys))))


def sv_last_error(h: int) -> str:
    return load_library().sv_last_error(ctypes.c_void_p(h)).decode()


def sv_last_stats(h: int) -> dict:
    st = sv_stats()
    _check(h, load_library().sv_last_stats(ctypes.c_void_p(h), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in sv_stats._fields_}


def sv_set_timing(h: int, enable: bool) -> None:
    _check(h, load_library().sv_set_timing(ctypes.c_void_p(h), int(bool(enable))))


def sv_phase_times(h: int) -> dict:
    ms = (ctypes.c_double * len(PHASES))()
    ln = (ctypes.c_uint64 * len(PHASES))()
    _check(h, load_library().sv_phase_times(ctypes.c_void_p(h), ms, ln))
    return {name: (ms[i], int(ln[i])) for i, name in enumerate(PHASES)}


def sv_launch_count() -> int:
    return int(load_library().sv_launch_count())


def sv_transfer_bytes():
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    load_library().sv_transfer_bytes(ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def sv_peak_noalloc(prec: int, keys_ptr: int, amps_ptr: int, n: int, stream: int = 0):
    """Peak of a caller-owned device term list without any allocation
    (see include/sv.h).  keys_ptr / amps_ptr are device addresses."""
    k, p = ctypes.c_uint64(), ctypes.c_double()
    rc = load_library().sv_peak_noalloc(prec, ctypes.c_void_p(keys_ptr), ctypes.c_void_p(amps_ptr),
                                        ctypes.c_uint64(n), ctypes.c_void_p(stream), ctypes.byref(k),
                                        ctypes.byref(p))
    if rc != SV_OK:
        raise SVError(rc, "sv_peak_noalloc failed")
    return k.value, p.value


SEL_BINS = 2048
_M64 = (1 << 64) - 1


def sv_select_histogram(h: int, prefix: int, bits: int):
    """Counts (uint32[2048]) and exact fixed-point masses (Python ints, in
    units of 2^-120) per value of the next digit of the composite
    Z = (~prob_bits, natural key) among the terms whose top `bits` bits of Z
    equal those of `prefix` (a 128-bit int)."""
    counts = np.zeros(SEL_BINS, dtype=np.uint32)
    masses = np.zeros(2 * SEL_BINS, dtype=np.uint64)
    _check(h, load_library().sv_select_histogram(ctypes.c_void_p(h), ctypes.c_uint64(prefix >> 64),
                                                 ctypes.c_uint64(prefix & _M64), int(bits),
                                                 counts.ctypes.data, masses.ctypes.data))
    hi, lo = masses[0::2], masses[1::2]
    return counts, [(int(a) << 64) | int(b) for a, b in zip(hi, lo)]


def sv_reserve(h: int, terms: int) -> None:
    """Size the handle's device buffers for states of up to `terms` terms."""
    _check(h, load_library().sv_reserve(ctypes.c_void_p(h), ctypes.c_uint64(int(terms))))


def sv_cut(h: int, z: int, S_c: int, S_N: int) -> int:
    """Keep the terms with composite Z <= z, renormalised by the kept mass
    S_c of all the handles together; S_N is their total mass (both exact
    fixed-point ints).  Returns this handle's term count."""
    kept = ctypes.c_uint64()
    _check(h, load_library().sv_cut(ctypes.c_void_p(h), ctypes.c_uint64(z >> 64), ctypes.c_uint64(z & _M64),
                                    ctypes.c_uint64(S_c >> 64), ctypes.c_uint64(S_c & _M64),
                                    ctypes.c_uint64(S_N >> 64), ctypes.c_uint64(S_N & _M64), ctypes.byref(kept)))
    return kept.value


def sv_probe_fp64(iters: int = 1 << 16, blocks_per_sm: int = 4):
    """FP64 fused multiply-add throughput of the current device: (TFLOP/s, ms)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = load_library().sv_probe_fp64(ctypes.c_uint64(iters), blocks_per_sm, ctypes.byref(tf), ctypes.byref(ms))
    if rc != 0:
        raise SVError(rc, "sv_probe_fp64 failed")
    return tf.value, ms.value


def sv_selftest(which: int, n: int, seed: int = 1):
    """Device self-test of the conversion-free complex64 arithmetic against
    the conversion instructions (see include/sv.h): returns (mismatches,
    first bad case index or None)."""
    bad, first = ctypes.c_uint64(), ctypes.c_uint64()
    rc = load_library().sv_selftest(which, ctypes.c_uint64(n), ctypes.c_uint64(seed), ctypes.byref(bad),
                                    ctypes.byref(first))
    if rc != SV_OK:
        raise SVError(rc, "sv_selftest failed")
    return bad.value, (None if first.value == (1 << 64) - 1 else first.value)


def sv_set_apply_variant(h: int, variant: int) -> None:
    _check(h, load_library().sv_set_apply_variant(ctypes.c_void_p(h), int(variant)))


# ------------------------------------------------ convenience wrapper
class SparseState:
    """A device-resident sparse state: keys u64, amplitudes complex128
    (``prec=SV_C128``) or complex64 with FP64 mass (``prec=SV_C64``)."""

    def __init__(self, n: int, K: int = 1 << 62, p: float = 1.0, prec: int = SV_C128, stream: int = 0):
        self.n, self.K, self.p, self.prec = n, int(K), float(p), prec
        self.h = sv_create_ex(n, int(K), float(p), prec, stream)

    def close(self):
        if getattr(self, "h", None):
            sv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_gate(self, qubits, u):
        sv_apply_gate(self.h, qubits, u)

    def truncate(self):
        return sv_truncate(self.h)

    def peak(self):
        return sv_peak(self.h)

    def peak_async(self) -> int:
        """Enqueue the peak readout and return a ticket at once; peak_wait
        returns the (key, probability) the state had at this call."""
        return sv_peak_async(self.h)

    def peak_wait(self, ticket: int):
        return sv_peak_wait(self.h, ticket)

    def num_terms(self) -> int:
        return sv_num_terms(self.h)

    def retained_mass(self) -> float:
        return sv_retained_mass(self.h)

    def probs(self):
        return sv_probs(self.h)

    def export(self):
        return sv_export(self.h)

    def load(self, keys, amps):
        sv_load(self.h, keys, amps)

    def stats(self) -> dict:
        return sv_last_stats(self.h)

    def set_timing(self, enable: bool = True) -> None:
        sv_set_timing(self.h, enable)

    def set_variant(self, variant: int) -> None:
        """0: group-first with grouping by partition and merge (default),
        1: expand-first, 2: group-first with a full radix sort (see
        include/sv.h)."""
        sv_set_apply_variant(self.h, variant)

    def phase_times(self) -> dict:
        return sv_phase_times(self.h)

    def reserve(self, terms: int) -> None:
        """Size the device buffers for states of up to `terms` terms (no
        allocation in later gates and truncations)."""
        sv_reserve(self.h, terms)

    def select_histogram(self, prefix: int, bits: int):
        return sv_select_histogram(self.h, prefix, bits)

    def cut(self, z: int, S_c: int, S_N: int) -> int:
        return sv_cut(self.h, z, S_c, S_N)

    def run(self, gates, truncate: bool = True):
        for (q, u) in gates:
            self.apply_gate(q, u)
            if truncate:
                self.truncate()
        return self


# ------------------------------------------------ batched form (svb_*)
def _bcheck(h, rc):
    if rc != SV_OK:
        raise SVError(rc, _lib.svb_last_error(h).decode() if h else "")


def svb_create(max_slots: int, prec: int = SV_C64, stream: int = 0) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    _bcheck(None, lib.svb_create(max_slots, prec, ctypes.c_void_p(stream), None, ctypes.byref(h)))
    return h.value


def svb_destroy(h: int) -> None:
    load_library().svb_destroy(ctypes.c_void_p(h))


def svb_add(h: int, n: int, K: int, p: float = 1.0) -> int:
    s = ctypes.c_int()
    _bcheck(h, load_library().svb_add(ctypes.c_void_p(h), n, ctypes.c_uint64(K), p, ctypes.byref(s)))
    return s.value


def svb_remove(h: int, slot: int) -> None:
    _bcheck(h, load_library().svb_remove(ctypes.c_void_p(h), slot))


# numpy layout of svb_gate (slot, m, qubits[4], U pointer): 32 bytes
GATE_DTYPE = np.dtype([("slot", "<i4"), ("m", "<i4"), ("q", "<i4", (4,)), ("U", "<u8")])
assert GATE_DTYPE.itemsize == ctypes.sizeof(svb_gate)


class PreparedGates:
    """A circuit's gates in the svb_gate layout, converted once: m, qubits
    and the address of each U inside one float64 buffer (kept alive here)."""

    def __init__(self, gates):
        gates = list(gates)
        self.count = len(gates)
        self.m = np.array([len(q) for q, _ in gates], dtype=np.int32)
        self.q = np.zeros((self.count, 4), dtype=np.int32)
        sizes = np.array([2 << (2 * int(m)) for m in self.m], dtype=np.int64)
        offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]) if self.count else np.zeros(0, np.int64)
        self.buf = np.empty(int(sizes.sum()) if self.count else 1, dtype=np.float64)
        for i, (q, u) in enumerate(gates):
            self.q[i, :len(q)] = q
            self.buf[offs[i]:offs[i] + sizes[i]] = _u_buffer(u)
        self.uptr = (self.buf.ctypes.data + 8 * offs).astype(np.uint64)


def svb_step_table(h: int, table: np.ndarray) -> None:
    """One step from a GATE_DTYPE array (its U addresses must stay valid
    for the call)."""
    table = np.ascontiguousarray(table, dtype=GATE_DTYPE)
    _bcheck(h, load_library().svb_step(ctypes.c_void_p(h), ctypes.c_void_p(table.ctypes.data), len(table)))


def svb_step(h: int, gates) -> None:
    """gates: iterable of (slot, qubits, U)."""
    gates = list(gates)
    arr = (svb_gate * max(1, len(gates)))()
    keep = []
    for i, (slot, q, u) in enumerate(gates):
        ub = _u_buffer(u)
        keep.append(ub)
        arr[i].slot = slot
        arr[i].m = len(q)
        for t, x in enumerate(q):
            arr[i].qubits[t] = int(x)
        arr[i].U = ub.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _bcheck(h, load_library().svb_step(ctypes.c_void_p(h), ctypes.cast(arr, ctypes.c_void_p), len(gates)))


def svb_num_terms(h: int, slot: int) -> int:
    n = ctypes.c_uint64()
    _bcheck(h, load_library().svb_num_terms(ctypes.c_void_p(h), slot, ctypes.byref(n)))
    return n.value


def svb_retained_mass(h: int, slot: int) -> float:
    f = ctypes.c_double()
    _bcheck(h, load_library().svb_retained_mass(ctypes.c_void_p(h), slot, ctypes.byref(f)))
    return f.value


def svb_peak(h: int, slot: int):
    k, p = ctypes.c_uint64(), ctypes.c_double()
    _bcheck(h, load_library().svb_peak(ctypes.c_void_p(h), slot, ctypes.byref(k), ctypes.byref(p)))
    return k.value, p.value


def svb_export(h: int, slot: int):
    n = svb_num_terms(h, slot)
    keys = np.zeros(n, dtype=np.uint64)
    amps = np.zeros(2 * n, dtype=np.float64)
    cnt = ctypes.c_uint64()
    _bcheck(h, load_library().svb_export(ctypes.c_void_p(h), slot, keys.ctypes.data, amps.ctypes.data,
                                         ctypes.c_uint64(n), ctypes.byref(cnt)))
    return keys, amps.view(np.complex128)


def svb_last_error(h: int) -> str:
    return load_library().svb_last_error(ctypes.c_void_p(h)).decode()


def svb_set_autotune(h: int, on: bool) -> None:
    _bcheck(h, load_library().svb_set_autotune(ctypes.c_void_p(h), 1 if on else 0))


def svb_set_graphs(h: int, on: bool) -> None:
    _bcheck(h, load_library().svb_set_graphs(ctypes.c_void_p(h), 1 if on else 0))


def svb_set_layer_kernel(h: int, on: bool) -> None:
    _bcheck(h, load_library().svb_set_layer_kernel(ctypes.c_void_p(h), 1 if on else 0))


def svb_peak_async(h: int, slot: int) -> int:
    t = ctypes.c_uint64()
    _bcheck(h, load_library().svb_peak_async(ctypes.c_void_p(h), slot, ctypes.byref(t)))
    return t.value


def svb_peak_wait(h: int, ticket: int):
    """(key, probability, retained mass) of a readout from svb_peak_async."""
    k, p, f = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
    _bcheck(h, load_library().svb_peak_wait(ctypes.c_void_p(h), ctypes.c_uint64(ticket), ctypes.byref(k),
                                            ctypes.byref(p), ctypes.byref(f)))
    return k.value, p.value, f.value


LAYER_PHASES = ["setup", "keys", "counts", "offsets", "scatter", "splits", "merge", "heads", "apply",
                "init", "pick1", "hist", "pick", "finish", "scale", "trunc"]


def svb_layer_phase_times(h: int):
    """Milliseconds per phase of the one-launch step, summed over the steps."""
    lib = load_library()
    arr = (ctypes.c_double * len(LAYER_PHASES))()
    cnt = ctypes.c_int()
    _bcheck(h, lib.svb_layer_phase_times(ctypes.c_void_p(h), arr, len(LAYER_PHASES), ctypes.byref(cnt)))
    return dict(zip(LAYER_PHASES, [float(x) for x in arr[:cnt.value]]))


def svb_graph_stats(h: int):
    c, n = ctypes.c_uint64(), ctypes.c_uint64()
    _bcheck(h, load_library().svb_graph_stats(ctypes.c_void_p(h), ctypes.byref(c), ctypes.byref(n)))
    return {"captures": c.value, "launches": n.value}


def svb_autotune_stats(h: int):
    t, c, d = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _bcheck(h, load_library().svb_autotune_stats(ctypes.c_void_p(h), ctypes.byref(t), ctypes.byref(c),
                                                 ctypes.byref(d)))
    return {"trials": t.value, "classes": c.value, "settled": d.value}


class Batch:
    """Many circuits advanced together (segmented state on the device)."""

    def __init__(self, max_slots: int, prec: int = SV_C64, stream: int = 0):
        self.h = svb_create(max_slots, prec, stream)
        self.prec = prec

    def close(self):
        if getattr(self, "h", None):
            svb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, n: int, K: int) -> int:
        return svb_add(self.h, n, K, 1.0)

    def remove(self, slot: int) -> None:
        svb_remove(self.h, slot)

    def step(self, gates) -> None:
        svb_step(self.h, gates)

    def step_table(self, table: np.ndarray) -> None:
        svb_step_table(self.h, table)

    def num_terms(self, slot: int) -> int:
        return svb_num_terms(self.h, slot)

    def retained_mass(self, slot: int) -> float:
        return svb_retained_mass(self.h, slot)

    def peak(self, slot: int):
        return svb_peak(self.h, slot)

    def export(self, slot: int):
        return svb_export(self.h, slot)

    def set_autotune(self, on: bool) -> None:
        svb_set_autotune(self.h, on)

    def autotune_stats(self):
        return svb_autotune_stats(self.h)

    def set_graphs(self, on: bool) -> None:
        svb_set_graphs(self.h, on)

    def graph_stats(self):
        return svb_graph_stats(self.h)

    def set_layer_kernel(self, on: bool) -> None:
        svb_set_layer_kernel(self.h, on)

    def layer_phase_times(self):
        return svb_layer_phase_times(self.h)

    def peak_async(self, slot: int) -> int:
        return svb_peak_async(self.h, slot)

    def peak_wait(self, ticket: int):
        return svb_peak_wait(self.h, ticket)
