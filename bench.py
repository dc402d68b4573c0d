#!/usr/bin/env python
"""Benchmark: sparse-gate terms/s and HBM / FP64 roofline fraction.

Workload: the n=40 brickwork peaked circuit (8 layers of Haar SU(4) on
neighbouring pairs, the perturbed mirror with theta ~ N(0, 0.05), X on the
hidden string), top-K truncation to K = 2^24 terms after every gate, p = 1.
One step = apply the next gate + truncate + read the peak, on the state
already at K terms (the whole hot path: key transform, grouping sort, group
mat-vec with zero drop, select, renormalising compaction, argmax).

value   : sum of input terms over the timed steps / device time of the steps
          (CUDA events on the library's stream; state resident in HBM and
          larger than L2, so no flush is needed).
e2e     : the same metric for the whole circuit run through the C ABI from
          the host (create, every gate with its matrix copied from host
          memory, every truncation, the peak read back), host wall clock.
roofline: the dominant kernel's algorithmic bytes (or FP64 flops) per launch
          over its CUDA-event launch time, against MEASURED_PEAKS.json.

--impl reference times the CPU oracle (test infrastructure, the only
reference that exists for this paper) on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS, K_TERMS, LAYERS, SEED = 40, 1 << 24, 8, 1002
SM_COUNT, FP64_FMA_PER_SM_CLK = 148, 2      # B300 FP64: 2 DFMA / SM / clock (probe: 0.56 TFMA/s @ 1.94 GHz)
WORKLOAD = "n40 brickwork Haar-SU(4) x8 + perturbed mirror + X^s, top-K 2^24 per gate, p=1"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="c128", choices=["c128", "c64"])
    ap.add_argument("--K", type=int, default=K_TERMS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-c64", action="store_true")
    ap.add_argument("--no-ring", action="store_true", help="skip the ring u3/cz (fusion) leg")
    ap.add_argument("--no-ab", action="store_true", help="skip the group-first / expand-first comparison")
    ap.add_argument("--serve-requests", type=int, default=128,
                    help="requests of the serving stream measured (0: skip the serving leg)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2032))}
    return {"hbm_gbs": 6400.0, "src": "fallback", "sm_max_mhz": 2032.0}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"sv_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks
def dist_reduce(vals, op: str):
    """Element-wise max or sum of a list of floats over all ranks (the list
    unchanged without a process group).  NCCL groups reduce on the current
    CUDA device, gloo groups on the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()]


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(units_local: float, ms_local: float):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling, every rank runs its own replica)."""
    units = dist_reduce([units_local], "sum")[0]
    ms = dist_reduce([ms_local], "max")[0]
    return units / (ms / 1e3), units, ms


# ------------------------------------------------------------------ roofline
def phase_model(ph: str, totals: dict, prec: str, passes: int):
    """Algorithmic bytes and FP64 flops of one phase over the timed steps.
    S_a = amplitude bytes; per term: key 8 B, probability 8 B."""
    sa = 16 if prec == "c128" else 8
    n_in, n_pre, n_kept = totals["n_in"], totals["n_pre"], totals["n_kept"]
    if ph == "sort":     # count pass (8 B) + scatter and merge passes (read + write the packed key: 16 B)
        return {"bytes": (8 + 16 * passes) * n_in, "flops": 0.0}
    if ph == "keys":     # radix-sort variant only: read key, write sort key + index
        return {"bytes": 20 * n_in, "flops": 0.0}
    if ph == "apply":    # read grouped key + gathered amplitude per input; write key+amp+prob per candidate
        return {"bytes": (8 + sa) * totals["n_in_apply"] + (16 + sa) * totals["n_pre_apply"],
                "flops": totals["fp64_apply"]}
    if ph == "window":   # one streaming pass over the probabilities (+ window keys)
        return {"bytes": 8 * n_pre, "flops": 0.0}
    if ph == "select":   # histogram levels over the window terms
        return {"bytes": 16 * totals.get("window_terms", 0), "flops": 0.0}
    if ph == "compact":  # keep bit per candidate; read kept key + amp; write kept key, amp, prob
        return {"bytes": n_pre / 8 + (8 + sa) * n_kept + (16 + sa) * n_kept, "flops": 0.0}
    if ph == "peak":     # after a truncation: the compaction's per-block partials
        return {"bytes": 16 * 1184 * totals["steps"], "flops": 0.0}
    if ph == "heads":    # read the grouped keys (group records written: not counted)
        return {"bytes": 8 * n_in, "flops": 0.0}
    if ph == "local":    # read key + amplitude per input; write key + amp + prob per candidate
        return {"bytes": (8 + sa) * totals["n_in_local"] + (16 + sa) * totals["n_pre_local"],
                "flops": totals["fp64_local"]}
    return {"bytes": 0.0, "flops": 0.0}


def dense_dfma_per_gate(m: int, n_in: int) -> float:
    # every input term meets 2^m outputs, 4 fused multiply-adds each, plus
    # the probability (2 ops) of every candidate (counted by the caller)
    return n_in * (1 << m) * 4.0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300 import sv

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sv.load_library()
    peaks = measured_peaks()

    def run_prec(prec_name, K, steps, warmup, sample_clocks):
        prec = sv.SV_C128 if prec_name == "c128" else sv.SV_C64
        circ = C.brickwork_n40(seed=SEED + rank, layers=LAYERS, K=K)
        gates = circ.gates
        st = sv.SparseState(circ.n, K, 1.0, prec=prec, stream=stream.cuda_stream)
        gi = 0
        # ramp: run until the state is at K terms
        while gi < len(gates) and st.num_terms() < K:
            q, u = gates[gi]
            st.apply_gate(q, u)
            st.truncate()
            gi += 1
        for _ in range(warmup):
            q, u = gates[gi % len(gates)]
            st.apply_gate(q, u)
            st.truncate()
            st.peak()
            gi += 1
        torch.cuda.synchronize(dev)
        barrier()
        totals = {"n_in": 0, "n_pre": 0, "n_kept": 0, "select_levels": 0, "steps": steps,
                  "sort_passes": 0, "window_hits": 0, "window_terms": 0,
                  # per gate path: the sorted path (sort + group mat-vec) or the bucket-local kernel
                  "n_in_apply": 0, "n_pre_apply": 0, "fp64_apply": 0.0,
                  "n_in_local": 0, "n_pre_local": 0, "fp64_local": 0.0}
        clocks = ClockSampler(dev.index) if sample_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        l0 = sv.sv_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        loc0 = st.stats()["local_gates"]
        pending = None
        e0.record(stream)
        for _ in range(steps):
            q, u = gates[gi % len(gates)]
            gi += 1
            st.apply_gate(q, u)
            st.truncate()
            # the peak of every step, read back pipelined: its 16 bytes reach
            # the host while the next step runs, and the statistics are
            # gathered while the compaction and the readout are on the GPU
            ticket = st.peak_async()
            s1 = s2 = st.stats()
            if pending is not None:
                st.peak_wait(pending)
            pending = ticket
            path = "local" if s1["local_gates"] > loc0 else "apply"
            loc0 = s1["local_gates"]
            totals["n_in_" + path] += s1["n_in"]
            totals["n_pre_" + path] += s1["n_pre"]
            # FP64 pipe work of the mat-vec kernel, counted as 2 flops per operation:
            # complex128 runs 4 fused multiply-adds per (input, output) pair, and
            # every candidate's probability is a multiply + fma (complex64 runs
            # the mat-vec in FP32, so only the probabilities are FP64)
            fp64_ops = 2.0 * s1["n_pre"]
            if prec == sv.SV_C128:
                fp64_ops += dense_dfma_per_gate(len(q), s1["n_in"])
            totals["fp64_" + path] += 2.0 * fp64_ops
            totals["n_in"] += s1["n_in"]
            totals["n_pre"] += s1["n_pre"]
            totals["n_kept"] += s2["n_kept"]
            totals["sort_passes"] += s1["sort_passes"]
            totals["select_levels"] += s2["select_levels"]
            totals["window_hits"] += s2["window_hits"]
            totals["window_terms"] += s2["window_terms"]
        if pending is not None:
            st.peak_wait(pending)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        launches = sv.sv_launch_count() - l0
        ms = e0.elapsed_time(e1)
        clk = clocks.stop() if clocks else None
        barrier()
        rate, units_all, ms = whole_job_rate(totals["n_in"], ms)
        # the per-phase breakdown: as many more steps with CUDA events around
        # every phase (kept out of the timed loop above: the events sit
        # between kernels of a step and cost time of their own)
        st.set_timing(True)
        for _ in range(steps):
            q, u = gates[gi % len(gates)]
            gi += 1
            st.apply_gate(q, u)
            st.truncate()
            st.peak_wait(st.peak_async())
        torch.cuda.synchronize(dev)
        phases = st.phase_times()
        peak = st.peak()
        fin = st.stats()
        paths = {k: fin[k] for k in ("local_gates", "global_gates", "local_fallbacks")}
        st.close()
        return {"ms": ms, "totals": totals, "phases": phases, "launches": launches, "clocks": clk,
                "peak": peak, "hidden": circ.hidden, "paths": paths, "rate": rate, "units_all": units_all}

    main = run_prec(args.prec, args.K, args.steps, args.warmup, sample_clocks=True)
    res = {"main": main}
    if not args.no_c64 and args.prec == "c128":
        res["c64"] = run_prec("c64", args.K, args.steps, args.warmup, sample_clocks=False)
    if not args.no_e2e:
        res["e2e"] = run_e2e(args, rank, dev, stream)
    if args.serve_requests > 0:
        res["serving"] = run_serving(args, rank, dev, stream)
    if not args.no_ring:
        res["ring"] = run_ring(args, dev, stream)
    if not args.no_ab:
        res["variant_ab"] = run_variant_ab(args, rank, dev, stream)
    return res, peaks


def run_e2e(args, rank, dev, stream):
    import numpy as np
    import torch
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300 import sv

    circ = C.brickwork_n40(seed=SEED + rank, layers=LAYERS, K=args.K)
    prec = sv.SV_C128 if args.prec == "c128" else sv.SV_C64
    # host-resident inputs: the gate matrices in pinned host memory
    pinned = [(q, torch.from_numpy(np.ascontiguousarray(u)).pin_memory().numpy()) for (q, u) in circ.gates]
    torch.cuda.synchronize(dev)
    barrier()
    h0, d0 = sv.sv_transfer_bytes()
    t0 = time.perf_counter()
    st = sv.SparseState(circ.n, args.K, 1.0, prec=prec, stream=stream.cuda_stream)
    n_in = 0
    for (q, u) in pinned:
        n_in += st.num_terms()
        st.apply_gate(q, u)
        st.truncate()
    key, pr = st.peak()
    st.close()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    h1, d1 = sv.sv_transfer_bytes()
    g = len(pinned)
    barrier()
    rate, _, _ = whole_job_rate(n_in, wall * 1e3)
    return {"value": rate, "unit": "terms/s", "h2d_bytes_per_step": int((h1 - h0) / g),
            "d2h_bytes_per_step": int((d1 - d0) / g), "wall_s": wall, "gates": g,
            "peak_is_hidden": bool(key == circ.hidden), "peak_prob": pr}


def run_serving(args, rank, dev, stream):
    """Serving form against the serial plain path on the same requests.

    Requests: the first R of the seeded serving stream (mirrored brickwork
    circuits, n in [16,48], forward depth in [2,10], K = 2^k with k in
    [10,20], and a 2% share of large ones with n=56, depth 12, K=2^25).
    serial  : each request alone on the single-state complex128 path, one
              after the other (create, every gate + top-k, peak, destroy);
              the service time of every request is measured.
    batched : the continuous-batching loop on the complex64 batched form,
              160 GB admission budget: a saturated run (all requests at t=0)
              gives the capacity; then a Poisson stream at 80% of it gives
              arrival-to-peak latencies.  The serial latencies at the same
              arrival times follow from its measured service times (one
              FIFO server)."""
    import numpy as np
    import torch
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300 import serve, sv

    R = args.serve_requests
    reqs = [C.serving_request(j) for j in range(R)]
    n_max = max(c.n for c in reqs)
    sv_stream = stream.cuda_stream
    torch.cuda.synchronize(dev)
    # warm-up of both paths on a few small requests
    small = [c for c in reqs if c.K <= 1 << 12][:4]
    serve.serve_serial_plain(small, prec=sv.SV_C128, stream=sv_stream)
    w = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=sv_stream)
    w.run(small)
    w.close()
    torch.cuda.synchronize(dev)

    t0 = time.perf_counter()
    ser = serve.serve_serial_plain(reqs, prec=sv.SV_C128, stream=sv_stream)
    torch.cuda.synchronize(dev)
    serial_s = time.perf_counter() - t0
    svc = np.array([x[0] for x in ser])

    srv = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=sv_stream)
    t0 = time.perf_counter()
    closed = srv.run(reqs)
    torch.cuda.synchronize(dev)
    closed_s = time.perf_counter() - t0
    steps_closed, resident = srv.steps, srv.peak_resident
    srv.close()
    fin = np.sort([r.finished for r in closed])
    lo, hi = fin[len(fin) // 4], fin[(3 * len(fin)) // 4]
    mid_rate = ((3 * len(fin)) // 4 - len(fin) // 4) / (hi - lo) if hi > lo else None
    capacity = R / closed_s
    rate = 0.8 * capacity
    arrivals = serve.poisson_arrivals(R, rate, 1005)
    srv = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=sv_stream)
    t0 = time.perf_counter()
    opened = srv.run(reqs, arrivals=arrivals)
    torch.cuda.synchronize(dev)
    open_s = time.perf_counter() - t0
    srv.close()
    p50, p99 = serve.percentiles(opened)
    s_lat = serve.fifo_latencies(arrivals, svc)
    same_peak = sum(int(a.peak_key == b[1]) for a, b in zip(closed, ser))
    # where the argmax differs, the two peak probabilities (complex64 batched,
    # complex128 serial): near-equal values mean a near-tie between strings
    differ = [(a.peak_prob, b[2]) for a, b in zip(closed, ser) if a.peak_key != b[1]]
    rel = [abs(x - y) / max(x, y) for x, y in differ]
    same_open = sum(int(a.peak_key == b.peak_key and a.peak_prob == b.peak_prob) for a, b in zip(opened, closed))
    large = [j for j, c in enumerate(reqs) if c.n == 56]
    return {
        "requests": R, "large_requests": len(large), "budget_gb": 160, "prec": "c64 batched vs c128 serial",
        "serial": {"circuits_per_s": R / svc.sum(), "wall_s": serial_s,
                   "p50_s": float(np.percentile(s_lat, 50)), "p99_s": float(np.percentile(s_lat, 99)),
                   "service_ms_p50": float(np.percentile(svc, 50) * 1e3)},
        "batched_closed": {"circuits_per_s": capacity, "wall_s": closed_s, "steps": steps_closed,
                           "max_resident": resident, "mid_run_circuits_per_s": mid_rate},
        "served": {"arrival_rate": rate, "circuits_per_s": R / (max(r.finished for r in opened) - arrivals[0]),
                   "p50_s": p50, "p99_s": p99, "wall_s": open_s},
        "speedup_circuits_per_s": capacity / (R / svc.sum()),
        "peaks_equal_to_serial_c128": f"{same_peak}/{R}",
        "differing_peaks_max_rel_prob_gap": max(rel) if rel else 0.0,
        "differing_peaks_max_prob": max((max(x, y) for x, y in differ), default=0.0),
        "served_results_equal_to_saturated_run": f"{same_open}/{R}",
    }


def run_variant_ab(args, rank, dev, stream, steps=8):
    """Group-first (default: grouping by partition and merge) against
    group-first with a full radix sort and against expand-first (the paper's
    formulation: one record per term and output, sorted, then summed per
    output) on the benchmark state at K terms: the same gates, alternating
    blocks of steps, CUDA-event time per step (gate + truncation) on the
    library's stream."""
    import torch
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300 import sv

    circ = C.brickwork_n40(seed=SEED + rank, layers=LAYERS, K=args.K)
    st = sv.SparseState(circ.n, args.K, 1.0, prec=sv.SV_C128, stream=stream.cuda_stream)
    gi = 0
    while gi < len(circ.gates) and st.num_terms() < args.K:
        q, u = circ.gates[gi]
        st.apply_gate(q, u)
        st.truncate()
        gi += 1
    ms = {0: [], 1: [], 2: []}
    for rep in range(2):
        for variant in (0, 2, 1):
            st.set_variant(variant)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps // 2):
                q, u = circ.gates[gi % len(circ.gates)]
                gi += 1
                st.apply_gate(q, u)
                st.truncate()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms[variant].append(e0.elapsed_time(e1) / (steps // 2))
    st.close()
    g, e, r = statistics.mean(ms[0]), statistics.mean(ms[1]), statistics.mean(ms[2])
    return {"K": args.K, "steps_each": steps, "group_first_ms_per_step": round(g, 3),
            "group_first_radix_sort_ms_per_step": round(r, 3),
            "expand_first_ms_per_step": round(e, 3), "expand_over_group": round(e / g, 3),
            "radix_over_merge_grouping": round(r / g, 3)}


def run_ring(args, dev, stream):
    """The ring-connected u3/cz workload shaped like the paper's example
    (44 qubits, 93 (u3, u3, cz) blocks walking the ring, their perturbed
    mirror, X on a seeded hidden string: about 580 instructions), run whole
    through the single-state complex128 path as given, after reordering and
    fusion into 2-qubit blocks (one update and truncation per block), and
    fused into blocks of up to 4 qubits: gates or blocks, wall time, and
    whether the peak is the hidden string."""
    import torch
    from paper_2607_07816_b300 import fusion, qasm, sv

    c = qasm.sharp_peak_circuit(n=44, blocks=93, K=32)
    variants = {"as_given": c.gates, "reordered_fused2": fusion.prepare(c.gates, 2),
                "fused4": fusion.fuse(c.gates, 4)}
    out = {"instructions": len(c.gates)}
    for K in (32, 1 << 10):
        for name, gates in variants.items():
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            st = sv.SparseState(c.n, K, 1.0, prec=sv.SV_C128, stream=stream.cuda_stream)
            for (q, u) in gates:
                st.apply_gate(q, u)
                st.truncate()
            key, pr = st.peak()
            F = st.retained_mass()
            st.close()
            torch.cuda.synchronize(dev)
            out[f"{name}_K{K}"] = {"updates": len(gates), "wall_ms": round(1e3 * (time.perf_counter() - t0), 2),
                                   "peak_is_hidden": bool(key == c.hidden), "peak_prob": pr,
                                   "retained_mass": F}
    return out


def roofline(main, prec, peaks):
    tot = main["totals"]
    phases = main["phases"]
    dom = max((p for p in phases if p != "other"), key=lambda p: phases[p][0])
    ms, launches = phases[dom]
    per_launch_s = ms / 1e3 / max(1, launches)
    passes = tot["sort_passes"] / max(1, tot["steps"])
    model = phase_model(dom, tot, prec, passes if dom == "sort" else 1)
    bytes_per_launch = model["bytes"] / max(1, launches)
    gbs = bytes_per_launch / per_launch_s / 1e9
    hbm_frac = gbs / peaks["hbm_gbs"]
    out = {"kernel": dom, "bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": round(hbm_frac, 4), "traffic": traffic_for(dom, bytes_per_launch),
           "peak_src": f"{peaks['src']} copy bandwidth", "launch_ms": round(per_launch_s * 1e3, 4),
           "launches": launches}
    if model["flops"] > 0:
        fp64_peak = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        tflops = model["flops"] / max(1, launches) / per_launch_s / 1e12
        if tflops / fp64_peak > hbm_frac:
            out.update({"bound": "alu", "achieved": round(tflops, 4), "peak": round(fp64_peak, 4),
                        "unit": "TFLOP/s", "frac": round(tflops / fp64_peak, 4),
                        "peak_src": "FP64 pipe: 148 SMs x 2 DFMA/clk x 2 flop x max SM clock",
                        "hbm_frac": round(hbm_frac, 4)})
    return out


def traffic_for(kernel, alg_bytes):
    """DRAM bytes per launch from the committed ncu summary, when it was
    taken on the current kernel sources (else null)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        from paper_2607_07816_b300 import build as B
        if d.get("source_hash") != B.source_hash():
            return None
        ent = d["kernels"].get(kernel)
        if not ent:
            return None
        return ent["dram_bytes_per_unit"] * ent["units_per_launch_full"]
    except Exception:
        return None


def gate_bytes_method(tot, prec):
    sa = 16 if prec == "c128" else 8
    S = 8 + sa
    b = 2 * S * tot["n_in"] + S * (tot["n_in"] + tot["n_pre"]) + 8 * tot["n_pre"] + S * (tot["n_pre"] + tot["n_kept"])
    strict = S * (tot["n_in"] + tot["n_kept"])
    return b, strict


# ------------------------------------------------------------------ CPU / reference arm
def oracle_sample(seconds: float, K_cap: int, max_gates: int = 10 ** 9):
    """The oracle as it stands, single-threaded, on the same circuit from
    |0...0>, gate after gate until `seconds` of CPU work have elapsed."""
    import oracle
    from paper_2607_07816_b300 import circuits as C
    circ = C.brickwork_n40(seed=SEED, layers=LAYERS, K=K_cap)
    o = oracle.Oracle(circ.n, K_cap, 1.0)
    n_in, g = 0, 0
    t0 = time.perf_counter()
    last = 0.0
    while g < min(len(circ.gates), max_gates):
        # stop before a gate that would overrun the budget (each brickwork
        # gate can multiply the term count by 4 until K is reached)
        if g > 0 and time.perf_counter() - t0 + 4.5 * last > seconds:
            break
        tg = time.perf_counter()
        q, u = circ.gates[g]
        n_in += o.num_terms()
        o.apply_gate(q, u)
        o.truncate()
        o.peak()
        g += 1
        last = time.perf_counter() - tg
    dt = time.perf_counter() - t0
    return {"value": n_in / dt, "unit": "terms/s", "cores": 1, "kind": "oracle",
            "sample": f"{WORKLOAD.split(',')[0]}: gates 1..{g} from |0>, K capped at {K_cap}, "
                      f"{n_in} input terms in {dt:.1f} s (single-threaded C++ std::map oracle)"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle  # noqa: F401  (builds the oracle if needed)
    per = []
    total_terms, total_t = 0, 0.0
    for i in range(args.warmup + args.steps):
        s = oracle_sample(seconds=1.0, K_cap=1 << 14, max_gates=40)
        if i >= args.warmup:
            per.append(s)
    vals = [p["value"] for p in per]
    v = statistics.mean(vals)
    line = {"metric": "sparse-gate terms/s", "value": v, "unit": "terms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n": N_QUBITS, "K": args.K, "p": 1.0, "prec": "c128"},
            "cpu_baseline": {"value": v, "unit": "terms/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: " + per[0]["sample"]},
            "e2e": {"value": v, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    res, peaks = run_ours(args, rank, world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    main_r = res["main"]
    tot = main_r["totals"]
    ms = main_r["ms"]
    value = main_r["rate"]
    bm, bstrict = gate_bytes_method(tot, args.prec)
    bw = peaks["hbm_gbs"] * 1e9
    line = {
        "metric": "sparse-gate terms/s", "value": value, "unit": "terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.prec == "c128" else "f32",
        "data": "synthetic (seeded Haar brickwork mirror circuit)",
        "config": {"workload": WORKLOAD, "n": N_QUBITS, "K": args.K, "p": 1.0, "prec": args.prec,
                   "layers": LAYERS, "seed": SEED, "l2": "state larger than L2 (no flush needed)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline(main_r, args.prec, peaks),
        "gate_roofline": {"B_method_frac": round(bm / (ms / 1e3) / bw, 4),
                          "B_strict_frac": round(bstrict / (ms / 1e3) / bw, 4),
                          "peak_gbs": peaks["hbm_gbs"]},
        "phases_ms": {k: round(v[0], 3) for k, v in main_r["phases"].items()},
        "phase_launches": {k: v[1] for k, v in main_r["phases"].items()},
        "gpu_launches": main_r["launches"],
        "clocks": main_r["clocks"],
        "peak_key": main_r["peak"][0],
        "totals": {k: (v if k.startswith("fp64") else int(v)) for k, v in tot.items()},
        "gate_paths": main_r.get("paths"),
    }
    if "c64" in res:
        c = res["c64"]
        ct = c["totals"]
        cb, _ = gate_bytes_method(ct, "c64")
        line["c64"] = {"value": c["rate"], "unit": "terms/s", "ms_per_step": c["ms"] / args.steps,
                       "B_method_frac": round(cb / (c["ms"] / 1e3) / bw, 4),
                       "roofline": roofline(c, "c64", peaks),
                       "phases_ms": {k: round(v[0], 3) for k, v in c["phases"].items()}}
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    if "serving" in res:
        line["serving"] = res["serving"]
    if "ring" in res:
        line["ring_u3cz"] = res["ring"]
    if "variant_ab" in res:
        line["apply_variant_ab"] = res["variant_ab"]
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = oracle_sample(seconds=15.0, K_cap=args.K)
        line["cpu_baseline"]["cores"] = 1
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
