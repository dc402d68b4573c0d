"""Textbook dense state-vector simulator used to pin the oracle.

A 2^n complex128 vector, each gate contracted over its qubits' tensor axes
(the dense representation the paper contrasts with, Sec. II).  It shares no
code with the oracle: it is an independent route to the same exact result.
"""
import numpy as np


def dense_zero(n: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    v[0] = 1.0
    return v


def dense_apply(psi: np.ndarray, n: int, qubits, u: np.ndarray) -> np.ndarray:
    m = len(qubits)
    t = psi.reshape((2,) * n)               # axis a <-> qubit n-1-a
    ut = np.asarray(u, dtype=np.complex128).reshape((2,) * (2 * m))
    # U's row/col index r has qubits[m-1] as most significant bit, so U axis j
    # (j < m) is local bit m-1-j, i.e. qubit qubits[m-1-j].
    in_axes = [n - 1 - qubits[m - 1 - j] for j in range(m)]
    out = np.tensordot(ut, t, axes=(list(range(m, 2 * m)), in_axes))
    # tensordot puts U's output axes first, then the untouched axes in order
    rest = [a for a in range(n) if a not in in_axes]
    order = in_axes + rest
    inv = np.argsort(order)
    return np.transpose(out, inv).reshape(-1)


def dense_run(n: int, gates) -> np.ndarray:
    psi = dense_zero(n)
    for (q, u) in gates:
        psi = dense_apply(psi, n, q, u)
    return psi
