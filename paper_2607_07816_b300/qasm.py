"""OpenQASM 2.0 front end and a ring-connected u3/cz circuit generator.

The paper's example workload (Sec. VI) is a circuit written in OpenQASM 2.0:
layers of single-qubit u3 rotations interleaved with cz gates between
neighbouring qubits of a 44-qubit chain closed into a ring (about 580
instructions).  This module reads such programs into the library's gate
list -- (qubits, U) with qubit i = key bit i, local index r = sum_t
bit(qubits[t]) << t, U row-major U[r_out][r_in], controls listed before the
target -- and writes gate lists back out, and it generates synthetic
circuits of the same shape (ring u3/cz blocks, mirrored with perturbed
inverses and closed by X on a seeded hidden string, so that the peak is
known).

Supported statements: OPENQASM, include, qreg, creg, measure and barrier
(the last three are skipped: the simulator reads out the peak) and the
gates u3, u2, u1, u, p,
rx, ry, rz, h, x, y, z, s, sdg, t, tdg, sx, sxdg, id, cx, cy, cz, ch, swap,
crz, cp / cu1, ccx and c3x.  Parameters are arithmetic expressions over
numbers and pi.
"""
from __future__ import annotations

import ast
import math
import re
from dataclasses import dataclass
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import circuits as C

Gate = Tuple[Tuple[int, ...], np.ndarray]


# ------------------------------------------------------------------ gate matrices
def mat_u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def _controlled(u: np.ndarray, controls: int) -> np.ndarray:
    """u on the last listed qubit, applied when every control is 1.  With
    controls listed first, they are the low bits of the local index."""
    d = 1 << (controls + 1)
    m = np.eye(d, dtype=np.complex128)
    cm = (1 << controls) - 1  # all control bits set
    i0, i1 = cm, cm | (1 << controls)  # target 0 / 1
    m[i0, i0], m[i0, i1] = u[0, 0], u[0, 1]
    m[i1, i0], m[i1, i1] = u[1, 0], u[1, 1]
    return m


def op_matrix(name: str, params: Sequence[float]) -> np.ndarray:
    p = list(params)
    if name in ("u3", "u"):
        return mat_u3(p[0], p[1], p[2])
    if name == "u2":
        return mat_u3(math.pi / 2, p[0], p[1])
    if name in ("u1", "p"):
        return np.diag([1.0, np.exp(1j * p[0])]).astype(np.complex128)
    if name == "rx":
        c, s = math.cos(p[0] / 2), math.sin(p[0] / 2)
        return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
    if name == "ry":
        c, s = math.cos(p[0] / 2), math.sin(p[0] / 2)
        return np.array([[c, -s], [s, c]], dtype=np.complex128)
    if name == "rz":
        return C.mat_rz(p[0])
    if name == "h":
        return C.mat_h()
    if name == "x":
        return C.mat_x()
    if name == "y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if name == "z":
        return np.diag([1.0, -1.0]).astype(np.complex128)
    if name == "s":
        return np.diag([1.0, 1j]).astype(np.complex128)
    if name == "sdg":
        return np.diag([1.0, -1j]).astype(np.complex128)
    if name == "t":
        return np.diag([1.0, np.exp(1j * math.pi / 4)]).astype(np.complex128)
    if name == "tdg":
        return np.diag([1.0, np.exp(-1j * math.pi / 4)]).astype(np.complex128)
    if name == "sx":
        return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
    if name == "sxdg":
        return 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]], dtype=np.complex128)
    if name == "id":
        return np.eye(2, dtype=np.complex128)
    if name == "cx":
        return C.mat_mcx(2)
    if name == "ccx":
        return C.mat_mcx(3)
    if name == "c3x":
        return C.mat_mcx(4)
    if name == "cy":
        return _controlled(op_matrix("y", []), 1)
    if name == "cz":
        return C.mat_cz()
    if name == "ch":
        return _controlled(C.mat_h(), 1)
    if name == "swap":
        return C.mat_swap()
    if name == "crz":
        return _controlled(C.mat_rz(p[0]), 1)
    if name in ("cp", "cu1"):
        return _controlled(op_matrix("p", p), 1)
    raise ValueError(f"unsupported gate {name}")


ARITY = {"u3": 1, "u": 1, "u2": 1, "u1": 1, "p": 1, "rx": 1, "ry": 1, "rz": 1, "h": 1, "x": 1, "y": 1,
         "z": 1, "s": 1, "sdg": 1, "t": 1, "tdg": 1, "sx": 1, "sxdg": 1, "id": 1, "cx": 2, "cy": 2, "cz": 2,
         "ch": 2, "swap": 2, "crz": 2, "cp": 2, "cu1": 2, "ccx": 3, "c3x": 4}
NPARAMS = {"u3": 3, "u": 3, "u2": 2, "u1": 1, "p": 1, "rx": 1, "ry": 1, "rz": 1, "crz": 1, "cp": 1, "cu1": 1}


@dataclass
class Op:
    """One instruction: gate name, parameters, global qubit indices."""
    name: str
    params: Tuple[float, ...]
    qubits: Tuple[int, ...]

    def gate(self) -> Gate:
        return (tuple(self.qubits), op_matrix(self.name, self.params))


# ------------------------------------------------------------------ expressions
_ALLOWED = (ast.Expression, ast.BinOp, ast.UnaryOp, ast.Constant, ast.Name, ast.Add, ast.Sub, ast.Mult,
            ast.Div, ast.Pow, ast.USub, ast.UAdd, ast.Load)


def eval_param(text: str) -> float:
    """An OpenQASM parameter: numbers, pi, + - * / ^ and parentheses."""
    tree = ast.parse(text.strip().replace("^", "**"), mode="eval")
    for node in ast.walk(tree):
        if not isinstance(node, _ALLOWED):
            raise ValueError(f"unsupported parameter expression: {text!r}")
        if isinstance(node, ast.Name) and node.id != "pi":
            raise ValueError(f"unknown name in parameter: {node.id}")
    return float(eval(compile(tree, "<param>", "eval"), {"__builtins__": {}}, {"pi": math.pi}))


def _split_params(s: str) -> List[str]:
    out, depth, cur = [], 0, ""
    for ch in s:
        if ch == "," and depth == 0:
            out.append(cur)
            cur = ""
            continue
        depth += ch == "("
        depth -= ch == ")"
        cur += ch
    if cur.strip():
        out.append(cur)
    return out


# ------------------------------------------------------------------ parser
_STMT = re.compile(r"^([a-z_][a-z0-9_]*)\s*(\((.*)\))?\s*(.*)$", re.I)
_QARG = re.compile(r"^([a-z_][a-z0-9_]*)\s*\[\s*(\d+)\s*\]$", re.I)


def parse(text: str) -> Tuple[int, List[Op]]:
    """Parse an OpenQASM 2.0 program: (number of qubits, instructions).
    Registers are laid out one after another in declaration order."""
    text = re.sub(r"//[^\n]*", "", text)
    regs: Dict[str, Tuple[int, int]] = {}
    nq = 0
    ops: List[Op] = []
    for raw in text.split(";"):
        st = raw.strip()
        if not st:
            continue
        low = st.lower()
        if low.startswith("openqasm") or low.startswith("include") or low.startswith("creg"):
            continue
        if low.startswith("measure") or low.startswith("barrier"):
            continue
        if low.startswith("qreg"):
            m = re.match(r"qreg\s+([a-z_][a-z0-9_]*)\s*\[\s*(\d+)\s*\]$", st, re.I)
            if not m:
                raise ValueError(f"bad qreg: {st}")
            regs[m.group(1)] = (nq, int(m.group(2)))
            nq += int(m.group(2))
            continue
        m = _STMT.match(st)
        if not m:
            raise ValueError(f"cannot parse: {st}")
        name = m.group(1).lower()
        if name not in ARITY:
            raise ValueError(f"unsupported gate {name}")
        params = tuple(eval_param(x) for x in _split_params(m.group(3))) if m.group(3) is not None else ()
        if len(params) != NPARAMS.get(name, 0):
            raise ValueError(f"{name} takes {NPARAMS.get(name, 0)} parameters: {st}")
        qs = []
        for a in [x.strip() for x in m.group(4).split(",") if x.strip()]:
            qm = _QARG.match(a)
            if not qm or qm.group(1) not in regs:
                raise ValueError(f"bad qubit argument {a!r} in {st}")
            off, size = regs[qm.group(1)]
            idx = int(qm.group(2))
            if idx >= size:
                raise ValueError(f"qubit index out of range in {st}")
            qs.append(off + idx)
        if len(qs) != ARITY[name] or len(set(qs)) != len(qs):
            raise ValueError(f"{name} needs {ARITY[name]} distinct qubits: {st}")
        ops.append(Op(name, params, tuple(qs)))
    return nq, ops


def dumps(n: int, ops: Sequence[Op]) -> str:
    """An OpenQASM 2.0 program for the instructions (one register q)."""
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg q[{n}];"]
    for op in ops:
        ps = "(" + ",".join(repr(float(x)) for x in op.params) + ")" if op.params else ""
        lines.append(f"{op.name}{ps} " + ",".join(f"q[{q}]" for q in op.qubits) + ";")
    return "\n".join(lines) + "\n"


def to_gates(ops: Sequence[Op]) -> List[Gate]:
    return [op.gate() for op in ops]


# ------------------------------------------------------------------ generator
def ring_edges(n: int) -> List[Tuple[int, int]]:
    """Neighbouring pairs 0-1, 1-2, ..., (n-2)-(n-1), then the wrap-around 0-(n-1)."""
    return [(i, i + 1) for i in range(n - 1)] + [(0, n - 1)]


def u3_inverse(params: Sequence[float]) -> Tuple[float, float, float]:
    """U3(t, f, l)^dagger = U3(-t, -l, -f)."""
    t, f, l = params
    return (-t, -l, -f)


def sharp_peak_like(n: int = 44, blocks: int = 93, seed: int = 1006, sigma: float = 0.05):
    """A ring-connected u3/cz circuit shaped like the paper's example: blocks
    (u3 on each qubit of a ring edge, then cz on the edge) walking the ring
    edges in order, then the mirror of those blocks with every u3 angle of
    the inverse perturbed by N(0, sigma), then X on the hidden string's
    one-bits (n = 44 and 93 blocks give about 580 instructions).  Returns
    (ops, hidden)."""
    rng = np.random.default_rng(seed)
    hidden = C.draw_hidden(n, rng)
    edges = ring_edges(n)
    fwd: List[Op] = []
    for b in range(blocks):
        a, c = edges[b % len(edges)]
        fwd.append(Op("u3", (float(rng.uniform(0, math.pi)), 0.0, -math.pi / 2), (a,)))
        fwd.append(Op("u3", (float(rng.uniform(0, math.pi)), 0.0, math.pi / 2), (c,)))
        fwd.append(Op("cz", (), (a, c)))
    inv: List[Op] = []
    for op in reversed(fwd):
        if op.name == "u3":
            t, f, l = u3_inverse(op.params)
            inv.append(Op("u3", (t + float(rng.normal(0, sigma)), f, l), op.qubits))
        else:
            inv.append(op)
    tail = [Op("x", (), (i,)) for i in range(n) if (hidden >> i) & 1]
    return fwd + inv + tail, hidden


def sharp_peak_circuit(n: int = 44, blocks: int = 93, seed: int = 1006, sigma: float = 0.05, K: int = 32,
                       p: float = 1.0) -> C.Circuit:
    ops, hidden = sharp_peak_like(n, blocks, seed, sigma)
    return C.Circuit(n=n, gates=to_gates(ops), hidden=hidden, K=K, p=p, name=f"ring_u3cz_n{n}")
