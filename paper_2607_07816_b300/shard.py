"""One state held across several GPUs (one handle per rank).

When K is beyond one GPU's memory (the device-memory wall of the paper's
performance section), the terms are partitioned by g "global" qubits over
W = 2^g ranks: rank r holds exactly the terms whose global qubits spell r
(bit j of r is the value of global qubit glob[j]).  Every term's key stays
complete, so each rank's handle is an ordinary state of the library.

* Gate on qubits that are all local: every rank applies it to its own terms
  (Eq. 3 only combines terms that differ in the gate's qubits, which all
  share the rank's global bits).
* Gate touching a global qubit glob[j]: that qubit first trades places with a
  local qubit l outside the gate.  Rank r keeps its terms whose bit l equals
  bit j of r and exchanges the others with rank r ^ 2^j, which does the
  same; afterwards glob[j] = l and the former global qubit is local.  One
  pairwise exchange per global qubit of the gate (a swap of partition bits).
* Truncation (Sec. III) over the union of the ranks' terms: a radix select
  on the canonical composite Z = (~prob bits, natural key), 11 bits per
  level, whose per-level histograms of counts and exact fixed-point masses
  (sv_select_histogram) are summed over the ranks; the top-k cut first, the
  p-mass cut only when the top-k kept mass reaches p of the total (then
  c_p <= K); every rank then keeps its terms up to the cut, renormalised by
  the global kept mass (sv_cut).  The result is the single-GPU rule applied
  to the whole state.
* Peak (Sec. V): the ranks' peaks reduced in canonical order.

Collectives run on the host through torch.distributed (a gloo group: the
histograms and the exchanged terms pass through host memory); each rank's
gate, histogram, compaction and renormalisation run in the library's kernels.
The per-rank engine is any object with the SparseState methods used here
(apply_gate, num_terms, export, load, select_histogram, cut, peak,
retained_mass), so the host logic can be tested with a stand-in engine.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Callable, List, Optional, Sequence

import numpy as np

TWO120 = 1 << 120
SEL_BITS = 11
_M32 = (1 << 32) - 1


def fx(v: float) -> int:
    """floor(v * 2^120) for a non-negative double, exactly."""
    return math.floor(Fraction(v) * TWO120) if v > 0 else 0


def fx_to_double(s: int) -> float:
    """The double nearest to s * 2^-120 (ties to even)."""
    return float(Fraction(s, TWO120))


class ShardedState:
    """A state of n qubits partitioned over the ranks of `group` (world size
    a power of two) by g = log2(world) global qubits, initially the top g
    qubits n-g .. n-1.  K and p are the truncation limits of the whole
    state.  make_engine(n) returns this rank's handle (a SparseState without
    its own truncation limits)."""

    def __init__(self, n: int, K: int, p: float, make_engine: Callable[[int], object], group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        g = self.world.bit_length() - 1
        if 1 << g != self.world:
            raise ValueError("the number of ranks must be a power of two")
        if g >= n:
            raise ValueError("more partition qubits than qubits")
        self.n, self.K, self.p = n, int(K), float(p)
        self.glob: List[int] = list(range(n - g, n))
        self.eng = make_engine(n)
        if self.rank != 0:  # |0...0> lives on the rank whose global bits are all zero
            self.eng.load(np.zeros(0, dtype=np.uint64), np.zeros(0, dtype=np.complex128))
        self.F = 1.0

    # ------------------------------------------------------------ collectives
    def _sum_ints(self, vals: Sequence[int]) -> List[int]:
        """Exact sum over the ranks of non-negative ints below 2^128 (as 32-bit
        limbs in int64 tensors, so no limb sum can overflow)."""
        import torch
        if self.world == 1:
            return [int(v) for v in vals]
        limbs = torch.tensor([[(int(v) >> (32 * k)) & _M32 for k in range(4)] for v in vals], dtype=torch.int64)
        self.dist.all_reduce(limbs, group=self.group)
        return [sum(int(x) << (32 * k) for k, x in enumerate(row)) for row in limbs.tolist()]

    def _gather_obj(self, obj):
        if self.world == 1:
            return [obj]
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out

    # ------------------------------------------------------------ gates
    def _swap_global(self, j: int, local: int) -> None:
        """Global qubit glob[j] trades places with local qubit `local`."""
        import torch
        mine = (self.rank >> j) & 1
        partner = self.rank ^ (1 << j)
        keys, amps = self.eng.export()
        bit = ((keys >> np.uint64(local)) & np.uint64(1)).astype(np.int64)
        stay = bit == mine
        out_k, out_a = keys[~stay], amps[~stay]
        # sizes first, then the terms (keys and interleaved re, im)
        cnt = torch.tensor([len(out_k)], dtype=torch.int64)
        rcnt = torch.zeros(1, dtype=torch.int64)
        reqs = [self.dist.isend(cnt, partner, group=self.group), self.dist.irecv(rcnt, partner, group=self.group)]
        for r in reqs:
            r.wait()
        m = int(rcnt.item())
        recv_k = torch.zeros(m, dtype=torch.int64)
        recv_a = torch.zeros(2 * m, dtype=torch.float64)
        reqs = []
        if len(out_k):
            send_k = torch.from_numpy(out_k.view(np.int64).copy())
            send_a = torch.from_numpy(np.ascontiguousarray(out_a).view(np.float64).copy())
            reqs += [self.dist.isend(send_k, partner, group=self.group, tag=1),
                     self.dist.isend(send_a, partner, group=self.group, tag=2)]
        if m:
            reqs += [self.dist.irecv(recv_k, partner, group=self.group, tag=1),
                     self.dist.irecv(recv_a, partner, group=self.group, tag=2)]
        for r in reqs:
            r.wait()
        new_k = np.concatenate([keys[stay], recv_k.numpy().view(np.uint64)])
        new_a = np.concatenate([amps[stay], recv_a.numpy().view(np.complex128)])
        self.eng.load(new_k, new_a)
        self.glob[j] = local

    def _balanced_local(self, exclude: Sequence[int]) -> int:
        """The local qubit outside `exclude` whose value splits the whole
        state most evenly (so the ranks keep similar term counts)."""
        free = [q for q in range(self.n) if q not in exclude and q not in self.glob]
        if not free:
            raise ValueError("no local qubit outside the gate to trade with a global one")
        keys, _ = self.eng.export()
        ones = [int(np.count_nonzero((keys >> np.uint64(q)) & np.uint64(1))) for q in free]
        tot = self._sum_ints(ones + [len(keys)])
        N = tot[-1]
        return min(zip(free, tot[:-1]), key=lambda qc: (abs(2 * qc[1] - N), qc[0]))[0]

    def apply_gate(self, qubits: Sequence[int], u) -> None:
        qs = [int(q) for q in qubits]
        for j, gq in enumerate(list(self.glob)):
            if gq in qs:
                self._swap_global(j, self._balanced_local(qs))
        self.eng.apply_gate(qs, u)

    # ------------------------------------------------------------ truncation
    def num_terms(self) -> int:
        return self._sum_ints([self.eng.num_terms()])[0]

    def _histogram(self, prefix: int, bits: int):
        counts, masses = self.eng.select_histogram(prefix, bits)
        tot = self._sum_ints([int(c) for c in counts] + list(masses))
        return tot[:len(counts)], tot[len(counts):]

    def _select(self, by_count: bool, target: int):
        """The cut of the radix select over all ranks: (Z_cut, c, S_c) where
        Z_cut bounds exactly the first c terms in canonical order, c the rank
        `target` (by count) or the smallest prefix whose mass reaches
        `target` (by mass); None when the mass target is never reached."""
        prefix, bits, before_c, before_m = 0, 0, 0, 0
        while True:
            counts, masses = self._histogram(prefix, bits)
            D = min(SEL_BITS, 128 - bits)
            chosen = None
            for d in range(1 << D):
                if by_count:
                    if before_c + counts[d] >= target:
                        chosen = d
                        break
                elif counts[d] and before_m + masses[d] >= target:
                    chosen = d
                    break
                before_c += counts[d]
                before_m += masses[d]
            if chosen is None:
                return None
            shift = 128 - bits - D
            prefix |= chosen << shift
            bits += D
            if counts[chosen] == 1 or bits == 128:
                # one term left in the bin: it is the cut; every Z up to the
                # bin's end bounds the same prefix of the canonical order
                z_cut = prefix | ((1 << shift) - 1)
                return z_cut, before_c + 1, before_m + masses[chosen]

    def truncate(self):
        """Sec. III over the whole state: c = min(c_p, K); returns (kept
        terms, retained fraction)."""
        N = self.num_terms()
        need_k, need_p = N > self.K, self.p < 1.0
        if N == 0 or not (need_k or need_p):
            return N, 1.0
        counts, masses = self._histogram(0, 0)
        S_N = sum(masses)
        T = fx(self.p * fx_to_double(S_N)) if need_p else None
        cut = None
        if need_k:
            cut = self._select(True, self.K)
            if need_p and cut[2] >= T:  # the mass cut lies at or before the K-th term
                cut = self._select(False, T)
        else:
            cut = self._select(False, T)
        if cut is None or cut[1] >= N:
            return N, 1.0
        z_cut, c, S_c = cut
        self.eng.cut(z_cut, S_c, S_N)
        f = fx_to_double(S_c) / fx_to_double(S_N)
        self.F *= f
        return c, f

    # ------------------------------------------------------------ readout
    def peak(self):
        """Most probable basis state of the whole state (probability
        descending, key ascending)."""
        mine = self.eng.peak() if self.eng.num_terms() else None
        cands = [x for x in self._gather_obj(mine) if x is not None]
        if not cands:
            raise ValueError("empty state")
        return min(cands, key=lambda kp: (-kp[1], kp[0]))

    def retained_mass(self) -> float:
        return self.F

    def export(self):
        """All ranks' terms (keys, amplitudes), rank after rank, on every
        rank."""
        keys, amps = self.eng.export()
        parts = self._gather_obj((keys, amps))
        k = np.concatenate([p[0] for p in parts]) if parts else np.zeros(0, dtype=np.uint64)
        a = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, dtype=np.complex128)
        return k, a

    def run(self, gates, truncate: bool = True):
        for (q, u) in gates:
            self.apply_gate(q, u)
            if truncate:
                self.truncate()
        return self
