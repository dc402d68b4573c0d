"""Sparsity-aware gate reordering and gate fusion (the front end of Sec. VI-B).

Two passes over a gate list (qubits, U), both leaving the circuit's unitary
unchanged:

* reorder: a topological order of the gate dependency graph (a gate depends
  on the previous gate on each of its qubits, so only gates on disjoint
  qubits change places) that keeps the set of active qubits -- qubits some
  earlier gate has acted on -- as small as possible: among the gates whose
  predecessors are all placed, one that touches only active qubits goes
  first (the earliest such), and only when there is none does the gate that
  brings in the fewest new qubits go next.  New qubits enter the state as
  late as the dependencies allow, which delays the growth of the number of
  nonzero terms.
* fuse: consecutive gates are merged into blocks acting on at most
  max_qubits qubits; each block becomes one unitary (the product of its
  gates, later gates on the left) on its qubits in ascending order.  The
  simulator then applies one update and one truncation per block instead of
  per gate.

With max_qubits = 2, a ring circuit of (u3, u3, cz) blocks fuses into one
two-qubit unitary per block, as in the paper; the engine takes up to 4.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

Gate = Tuple[Tuple[int, ...], np.ndarray]


def dependencies(gates: Sequence[Gate]) -> List[List[int]]:
    """preds[j]: the previous gate on each qubit of gate j."""
    last = {}
    preds = []
    for j, (q, _) in enumerate(gates):
        preds.append(sorted({last[x] for x in q if x in last}))
        for x in q:
            last[x] = j
    return preds


def reorder(gates: Sequence[Gate], active: Sequence[int] = ()) -> List[Gate]:
    """The gates in a dependency-respecting order that postpones new qubits
    (``active``: qubits already active before the first gate)."""
    gates = list(gates)
    preds = dependencies(gates)
    succs: List[List[int]] = [[] for _ in gates]
    waiting = [len(p) for p in preds]
    for j, p in enumerate(preds):
        for i in p:
            succs[i].append(j)
    ready = sorted(j for j in range(len(gates)) if waiting[j] == 0)
    act = set(active)
    out: List[Gate] = []
    while ready:
        pick = None
        for j in ready:  # ready is kept in original order
            if all(x in act for x in gates[j][0]):
                pick = j
                break
        if pick is None:
            pick = min(ready, key=lambda j: (sum(1 for x in gates[j][0] if x not in act), j))
        ready.remove(pick)
        out.append(gates[pick])
        act.update(gates[pick][0])
        for k in succs[pick]:
            waiting[k] -= 1
            if waiting[k] == 0:
                # insert keeping the original order
                lo, hi = 0, len(ready)
                while lo < hi:
                    mid = (lo + hi) // 2
                    if ready[mid] < k:
                        lo = mid + 1
                    else:
                        hi = mid
                ready.insert(lo, k)
    return out


def embed(q: Sequence[int], u: np.ndarray, block: Sequence[int]) -> np.ndarray:
    """The gate (q, u) as a unitary on the block's qubits (bit k of the block
    index is qubit block[k]; bit t of the gate index is qubit q[t])."""
    M = len(block)
    pos = [list(block).index(x) for x in q]
    gmask = sum(1 << p for p in pos)
    d = 1 << M
    E = np.zeros((d, d), dtype=np.complex128)
    for ri in range(d):
        gi = sum(((ri >> p) & 1) << t for t, p in enumerate(pos))
        rest = ri & ~gmask
        for go in range(1 << len(q)):
            ro = rest | sum(((go >> t) & 1) << p for t, p in enumerate(pos))
            E[ro, ri] = u[go, gi]
    return E


def fuse(gates: Sequence[Gate], max_qubits: int = 2) -> List[Gate]:
    """Merge runs of consecutive gates whose qubits together number at most
    max_qubits (1..4) into single unitaries."""
    if not 1 <= max_qubits <= 4:
        raise ValueError("max_qubits must be 1..4")
    out: List[Gate] = []
    run: List[Gate] = []
    qs: set = set()

    def close():
        if not run:
            return
        block = tuple(sorted(qs))
        U = np.eye(1 << len(block), dtype=np.complex128)
        for (q, u) in run:
            U = embed(q, np.asarray(u, dtype=np.complex128), block) @ U
        out.append((block, U))

    for (q, u) in gates:
        if len(q) > max_qubits:
            raise ValueError(f"a gate on {len(q)} qubits exceeds max_qubits={max_qubits}")
        if run and len(qs | set(q)) > max_qubits:
            close()
            run, qs = [], set()
        run.append((tuple(q), u))
        qs |= set(q)
    close()
    return out


def prepare(gates: Sequence[Gate], max_qubits: int = 2, reorder_first: bool = True) -> List[Gate]:
    """Reorder (optionally), then fuse: the block list the simulator runs."""
    g = reorder(gates) if reorder_first else list(gates)
    return fuse(g, max_qubits)


def active_profile(gates: Sequence[Gate]) -> List[int]:
    """Number of active qubits after each gate (how fast qubits come in)."""
    act: set = set()
    prof = []
    for (q, _) in gates:
        act.update(q)
        prof.append(len(act))
    return prof
