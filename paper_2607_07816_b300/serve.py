"""Serving form: continuous batching of circuit requests over the batched C ABI.

Requests (circuits) arrive over time.  The loop admits an arrived request
into a free slot of the device-resident batch whenever its footprint
(K * 2^m_max * 16 bytes, the most a gate can expand its state to) fits the
HBM budget next to the circuits already resident, advances every resident
circuit by one gate per step (one svb_step for all of them), and retires a
circuit as soon as its last gate has run: its most probable basis state
(Sec. V) is read back and its slot and budget are released for the next
arrivals.  Work of newly admitted and long-running circuits overlaps in the
same steps.

A request whose K reaches solo_min_terms is not batched: a state that large
fills the GPU by itself, so batching gains it nothing, while the single-state
engine groups its terms faster.  It is admitted against the same budget and
runs gate by gate on a handle and stream of its own, in a host thread, while
the batch keeps stepping; the two streams' kernels share the GPU.  The
result is bit for bit that of the same circuit alone on the single-state
engine.  The loop itself only orders requests and marshals gates; every
gate, truncation and readout runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from collections import deque
from typing import List, Optional, Sequence

import numpy as np

from . import sv


@dataclasses.dataclass
class Result:
    index: int
    peak_key: int
    peak_prob: float
    retained_mass: float
    arrival: float
    admitted: float
    finished: float
    keys: Optional[np.ndarray] = None
    amps: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint(circuit) -> int:
    """Admission size of a request: K * 2^m_max * 16 bytes, the most its
    state can grow to inside one gate before the cut (Sec. IV-A)."""
    m_max = max((len(q) for q, _ in circuit.gates), default=1)
    return int(circuit.K) * (1 << m_max) * 16


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def slot_limit(n_max: int, max_slots: int) -> int:
    """Most slots a batch may hold while a circuit of n_max qubits can still be
    admitted: the step's 64-bit sort key holds the slot index above the key."""
    bits = 64 - n_max
    return max(1, min(max_slots, (1 << bits) - 1))


def _new_stream():
    """A stream for a solo request (PyTorch supplies the CUDA streams)."""
    import torch
    return torch.cuda.Stream()


class Server:
    """A continuous-batching request loop on one GPU.

    budget_bytes bounds the sum of the resident requests' footprints;
    max_slots bounds how many are resident at once (lowered when n_max, the
    largest qubit count that will be served, needs more key bits).  Requests
    with K >= solo_min_terms run on single-state handles of their own, each
    on a stream from solo_stream() (an object with a cuda_stream handle)."""

    def __init__(self, budget_bytes: int, max_slots: int = 512, n_max: int = 54, prec: int = sv.SV_C64,
                 stream: int = 0, batch=None, solo_min_terms: int = 1 << 22, solo_stream=None,
                 one_launch: Optional[bool] = None):
        self.budget = int(budget_bytes)
        self.max_slots = slot_limit(n_max, max_slots)
        self.prec = prec
        self.batch = batch if batch is not None else sv.Batch(self.max_slots, prec=prec, stream=stream)
        if one_launch is not None:  # each step one persistent launch (steps then run ahead of the host)
            self.batch.set_layer_kernel(one_launch)
        self.solo_min_terms = int(solo_min_terms)
        self.solo_stream = solo_stream if solo_stream is not None else _new_stream
        self.steps = 0
        self.peak_resident = 0
        self.peak_bytes = 0
        self.solo_served = 0

    def close(self):
        self.batch.close()

    def run(self, circuits: Sequence, arrivals: Optional[Sequence[float]] = None, clock=None,
            export: bool = False, max_steps: Optional[int] = None) -> List[Result]:
        """Serve every circuit and return one Result per circuit, in input
        order.  arrivals[j] is when request j arrives, in the units of clock
        (seconds after the start by default; all 0 when None: a saturated
        run).  A request is admitted, in arrival order, once it has arrived,
        a slot is free and its footprint fits the budget (one request is
        always admitted into an empty batch).  With export the final state of
        each circuit is returned as well (export may also be a collection of
        request indices: only those are exported).  max_steps stops the loop
        after that many steps (unfinished requests then have no Result).

        Each admitted circuit's gates are converted once into the library's
        gate layout; the gate table of a step is then gathered with array
        indexing from the concatenated tables of the resident circuits
        (rebuilt only when residents change)."""
        n = len(circuits)
        if isinstance(export, bool):
            wants = (lambda j: export)  # noqa: E731
        else:
            chosen = set(int(j) for j in export)
            wants = chosen.__contains__
        arrivals = np.zeros(n) if arrivals is None else np.asarray(arrivals, dtype=float)
        if clock is None:
            t0 = time.perf_counter()
            clock = lambda: time.perf_counter() - t0  # noqa: E731
        order = deque(np.argsort(arrivals, kind="stable").tolist())
        results: List[Optional[Result]] = [None] * n
        live = {}  # slot -> [request index, next gate, admission time, prepared gates]
        used = 0
        retiring = 0  # slots removed since the last step (free after it)
        done = 0
        dirty = True
        slots = np.zeros(0, dtype=np.int32)
        pos = np.zeros(0, dtype=np.int64)
        solo_lock = threading.Lock()
        solo_finished: List = []  # (request index, Result or exception) from the solo threads
        solo_threads: List[threading.Thread] = []
        solo_running = 0
        inflight: List = []  # (request index, readout ticket, admission time) of retired slots

        def collect() -> int:
            """Results of the readouts enqueued so far (waits for each)."""
            got = 0
            for j, ticket, admitted in inflight:
                key, prob, f = self.batch.peak_wait(ticket)
                results[j] = Result(j, key, prob, f, float(arrivals[j]), admitted, clock())
                got += 1
            inflight.clear()
            return got

        def solo(j: int, c, admitted: float) -> None:
            try:
                stream = self.solo_stream()
                st = sv.SparseState(c.n, c.K, 1.0, prec=self.prec, stream=stream.cuda_stream)
                try:
                    for (q, u) in c.gates:
                        st.apply_gate(q, u)
                        st.truncate()
                    key, prob = st.peak()
                    f = st.retained_mass()
                    ks = am = None
                    if wants(j):
                        ks, am = st.export()
                finally:
                    st.close()
                out = Result(j, key, prob, f, float(arrivals[j]), admitted, clock(), ks, am)
            except BaseException as e:  # noqa: BLE001 - re-raised by the loop
                out = e
            with solo_lock:
                solo_finished.append((j, out))

        try:
            while done < n and (max_steps is None or self.steps < max_steps):
                now = clock()
                with solo_lock:
                    finished, solo_finished[:] = list(solo_finished), []
                for j, out in finished:
                    if isinstance(out, BaseException):
                        raise out
                    results[j] = out
                    used -= footprint(circuits[j])
                    solo_running -= 1
                    done += 1
                while order and arrivals[order[0]] <= now:
                    j = order[0]
                    c = circuits[j]
                    fp = footprint(c)
                    is_solo = c.K >= self.solo_min_terms and c.gates
                    if not is_solo and len(live) + retiring >= self.max_slots:
                        break  # wait for a slot
                    if used + fp > self.budget and (live or solo_running):
                        break  # wait for resident requests to finish
                    order.popleft()
                    if not c.gates:
                        results[j] = Result(j, 0, 1.0, 1.0, float(arrivals[j]), now, now)
                        done += 1
                        continue
                    used += fp
                    if is_solo:
                        t = threading.Thread(target=solo, args=(j, c, now), daemon=True)
                        solo_running += 1
                        self.solo_served += 1
                        solo_threads.append(t)
                        t.start()
                        continue
                    slot = self.batch.add(c.n, c.K)
                    live[slot] = [j, 0, now, sv.PreparedGates(c.gates)]
                    dirty = True
                self.peak_resident = max(self.peak_resident, len(live) + solo_running)
                self.peak_bytes = max(self.peak_bytes, used)
                if not live:
                    if inflight:
                        done += collect()
                        continue
                    if retiring:  # an empty step frees the retired slots
                        self.batch.step([])
                        retiring = 0
                    elif solo_running:  # only solo requests are running
                        time.sleep(0.0005)
                    elif order:  # idle until the next arrival
                        wait = arrivals[order[0]] - clock()
                        if wait > 0:
                            time.sleep(min(wait, 0.01))
                    continue
                if dirty:  # residents changed: concatenate their gate tables
                    for k, sl in enumerate(slots):  # positions of the circuits that stay
                        if int(sl) in live:
                            live[int(sl)][1] = int(pos[k])
                    slots = np.array(list(live), dtype=np.int32)
                    preps = [live[int(sl)][3] for sl in slots]
                    counts = np.array([p.count for p in preps], dtype=np.int64)
                    base = np.concatenate([[0], np.cumsum(counts)[:-1]])
                    tm = np.concatenate([p.m for p in preps])
                    tq = np.concatenate([p.q for p in preps])
                    tu = np.concatenate([p.uptr for p in preps])
                    pos = np.array([live[int(sl)][1] for sl in slots], dtype=np.int64)
                    table = np.empty(len(slots), dtype=sv.GATE_DTYPE)
                    table["slot"] = slots
                    dirty = False
                idx = base + pos
                table["m"] = tm[idx]
                table["q"] = tq[idx]
                table["U"] = tu[idx]
                self.batch.step_table(table)
                self.steps += 1
                retiring = 0
                pos += 1
                # the readouts of the slots retired after the previous step
                # complete while this step runs
                done += collect()
                for k in np.nonzero(pos == counts)[0]:
                    slot = int(slots[k])
                    j, _, admitted, _ = live[slot]
                    if wants(j):  # read at once, with the final state
                        key, prob = self.batch.peak(slot)
                        f = self.batch.retained_mass(slot)
                        ks, am = self.batch.export(slot)
                        results[j] = Result(j, key, prob, f, float(arrivals[j]), admitted, clock(), ks, am)
                        done += 1
                    else:  # pipelined: collected after the next step is enqueued
                        inflight.append((j, self.batch.peak_async(slot), admitted))
                    self.batch.remove(slot)
                    retiring += 1
                    del live[slot]
                    used -= footprint(circuits[j])
                    dirty = True
                if dirty:  # retirements: save the positions before a slot can be reused
                    for k, sl in enumerate(slots):
                        if int(sl) in live:
                            live[int(sl)][1] = int(pos[k])
                    slots = np.zeros(0, dtype=np.int32)
                    pos = np.zeros(0, dtype=np.int64)
        finally:
            for t in solo_threads:
                t.join()
        return results  # type: ignore[return-value]


def percentiles(results: Sequence[Result]):
    lat = np.array([r.latency for r in results])
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


def serve_serial_plain(circuits: Sequence, prec: int = sv.SV_C128, stream: int = 0,
                       clock=time.perf_counter):
    """The serial plain path: every circuit alone, one after the other, on
    the single-state API (gate, then top-k truncation, then the peak).
    Returns the service time of each circuit and its peak."""
    out = []
    for c in circuits:
        t = clock()
        st = sv.SparseState(c.n, c.K, 1.0, prec=prec, stream=stream)
        for (q, u) in c.gates:
            st.apply_gate(q, u)
            st.truncate()
        key, prob = st.peak()
        st.close()
        out.append((clock() - t, key, prob))
    return out


def fifo_latencies(arrivals: Sequence[float], service: Sequence[float]) -> np.ndarray:
    """Completion minus arrival of a single FIFO server with the given
    service times (the serial path cannot overlap circuits)."""
    t = 0.0
    lat = []
    for a, s in zip(arrivals, service):
        start = max(t, a)
        t = start + s
        lat.append(t - a)
    return np.array(lat)


def main(argv=None) -> None:
    """Serve a seeded synthetic request stream and print one JSON summary
    (python -m paper_2607_07816_b300.serve --help)."""
    import argparse
    import json

    from . import circuits as C

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--seed", type=int, default=1005)
    ap.add_argument("--large-frac", type=float, default=0.02)
    ap.add_argument("--k-min", type=int, default=10)
    ap.add_argument("--k-max", type=int, default=20)
    ap.add_argument("--rate", type=float, default=0.0, help="Poisson arrivals per second (0: all at t=0)")
    ap.add_argument("--prec", choices=["c64", "c128"], default="c64")
    ap.add_argument("--budget-gb", type=float, default=160.0)
    ap.add_argument("--max-steps", type=int, default=None)
    ap.add_argument("--form", choices=["one_launch", "kernels"], default="one_launch",
                    help="the batched step as one persistent launch, or as separate kernels")
    ap.add_argument("--no-autotune", action="store_true", help="fixed launch shapes (separate kernels)")
    a = ap.parse_args(argv)
    reqs = [C.serving_request(j, seed=a.seed, large_frac=a.large_frac, k_range=(a.k_min, a.k_max))
            for j in range(a.requests)]
    arrivals = poisson_arrivals(len(reqs), a.rate, a.seed) if a.rate > 0 else None
    srv = Server(int(a.budget_gb * (1 << 30)), n_max=max(c.n for c in reqs),
                 prec=sv.SV_C64 if a.prec == "c64" else sv.SV_C128, one_launch=a.form == "one_launch")
    if a.no_autotune:
        srv.batch.set_autotune(False)
    t0 = time.perf_counter()
    res = srv.run(reqs, arrivals=arrivals, max_steps=a.max_steps)
    wall = time.perf_counter() - t0
    fin = [r for r in res if r is not None]
    out = {"requests": len(reqs), "finished": len(fin), "steps": srv.steps, "wall_s": wall,
           "circuits_per_s": len(fin) / wall if wall > 0 else None, "max_resident": srv.peak_resident,
           "graphs": srv.batch.graph_stats(), "autotune": srv.batch.autotune_stats(), "form": a.form}
    if a.form == "one_launch":
        out["layer_phases_ms"] = {k: round(v, 3) for k, v in srv.batch.layer_phase_times().items()}
    if fin:
        lat = np.array([r.latency for r in fin])
        out.update({"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99))})
    srv.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
