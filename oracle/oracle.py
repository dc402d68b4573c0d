"""ctypes wrapper around the C++ oracle (``sv_oracle.cpp``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain single-threaded CPU
restatement of the paper's method (Sec. I-V): an ordered map of nonzero
amplitudes, the gate rule of Eq. (3) generalised to 2^m x 2^m, the p-mass and
top-k truncations of Sec. III with renormalisation, and the most-probable
readout of Sec. V.  It shares no code with the CUDA library and never
imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

C128, C64 = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE double semantics: no fast-math and
    no FP contraction beyond the explicit fma calls."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17",
                               "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            P = ctypes.POINTER
            lib.or_create.restype = vp
            lib.or_create.argtypes = [i32, u64, dbl, i32]
            lib.or_destroy.argtypes = [vp]
            lib.or_apply_gate.restype = i32
            lib.or_apply_gate.argtypes = [vp, i32, P(ctypes.c_int), P(dbl)]
            lib.or_truncate.restype = i32
            lib.or_truncate.argtypes = [vp, P(u64), P(dbl)]
            lib.or_peak.restype = i32
            lib.or_peak.argtypes = [vp, P(u64), P(dbl)]
            lib.or_num_terms.restype = u64
            lib.or_num_terms.argtypes = [vp]
            lib.or_retained_mass.restype = dbl
            lib.or_retained_mass.argtypes = [vp]
            lib.or_export.restype = i32
            lib.or_export.argtypes = [vp, vp, vp, vp, u64, P(u64)]
            lib.or_load.restype = i32
            lib.or_load.argtypes = [vp, vp, vp, u64]
            lib.or_total_mass_fx.argtypes = [vp, P(u64), P(u64)]
            lib.or_last_cut.argtypes = [vp] + [P(u64)] * 6
            lib.or_fx.argtypes = [dbl, P(u64), P(u64)]
            lib.or_fx_to_double.restype = dbl
            lib.or_fx_to_double.argtypes = [u64, u64]
            lib.or_prob.restype = dbl
            lib.or_prob.argtypes = [dbl, dbl]
            _lib = lib
    return _lib


def fx(p: float) -> int:
    """floor(p * 2^120) as a Python int (the oracle's fixed-point mass)."""
    lib = _load()
    hi, lo = ctypes.c_uint64(), ctypes.c_uint64()
    lib.or_fx(float(p), ctypes.byref(hi), ctypes.byref(lo))
    return (hi.value << 64) | lo.value


def fx_to_double(s: int) -> float:
    lib = _load()
    return lib.or_fx_to_double(ctypes.c_uint64(s >> 64), ctypes.c_uint64(s & (2**64 - 1)))


def prob(re: float, im: float) -> float:
    return _load().or_prob(float(re), float(im))


def _u_buffer(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.complex128))
    return u.view(np.float64).reshape(-1).copy()


class Oracle:
    """One oracle state (complex128 or complex64 form)."""

    def __init__(self, n: int, K: int = 1 << 62, p: float = 1.0, prec: int = C128):
        self._lib = _load()
        self.n, self.K, self.p, self.prec = n, int(K), float(p), prec
        self._h = self._lib.or_create(n, ctypes.c_uint64(int(K)), float(p), prec)
        if not self._h:
            raise ValueError("oracle: invalid arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    def apply_gate(self, qubits, u) -> None:
        m = len(qubits)
        q = (ctypes.c_int * m)(*[int(x) for x in qubits])
        ub = _u_buffer(u)
        rc = self._lib.or_apply_gate(self._h, m, q, ub.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if rc != 0:
            raise ValueError(f"oracle apply_gate failed ({rc})")

    def truncate(self):
        kept, f = ctypes.c_uint64(), ctypes.c_double()
        self._lib.or_truncate(self._h, ctypes.byref(kept), ctypes.byref(f))
        return kept.value, f.value

    def peak(self):
        k, pr = ctypes.c_uint64(), ctypes.c_double()
        rc = self._lib.or_peak(self._h, ctypes.byref(k), ctypes.byref(pr))
        if rc != 0:
            raise ValueError("oracle: empty state")
        return k.value, pr.value

    def num_terms(self) -> int:
        return int(self._lib.or_num_terms(self._h))

    def retained_mass(self) -> float:
        return float(self._lib.or_retained_mass(self._h))

    def export(self):
        """(keys uint64, amps complex128, probs float64) in canonical order
        (probability descending, key ascending)."""
        n = self.num_terms()
        keys = np.zeros(n, dtype=np.uint64)
        amps = np.zeros(2 * n, dtype=np.float64)
        probs = np.zeros(n, dtype=np.float64)
        cnt = ctypes.c_uint64()
        self._lib.or_export(self._h, keys.ctypes.data, amps.ctypes.data, probs.ctypes.data,
                            ctypes.c_uint64(n), ctypes.byref(cnt))
        return keys, amps.view(np.complex128), probs

    def load(self, keys, amps) -> None:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        a = np.ascontiguousarray(np.asarray(amps, dtype=np.complex128)).view(np.float64)
        rc = self._lib.or_load(self._h, keys.ctypes.data, a.ctypes.data, ctypes.c_uint64(len(keys)))
        if rc != 0:
            raise ValueError("oracle: invalid state")

    def total_mass_fx(self) -> int:
        hi, lo = ctypes.c_uint64(), ctypes.c_uint64()
        self._lib.or_total_mass_fx(self._h, ctypes.byref(hi), ctypes.byref(lo))
        return (hi.value << 64) | lo.value

    def last_cut(self):
        v = [ctypes.c_uint64() for _ in range(6)]
        self._lib.or_last_cut(self._h, *[ctypes.byref(x) for x in v])
        N, c, snh, snl, sch, scl = [x.value for x in v]
        return {"N": N, "c": c, "SN": (snh << 64) | snl, "Sc": (sch << 64) | scl}

    def run(self, gates, truncate: bool = True):
        """Apply each gate, truncating after every gate (the per-gate
        schedule of the workloads)."""
        for (q, u) in gates:
            self.apply_gate(q, u)
            if truncate:
                self.truncate()
        return self
