#!/usr/bin/env python
"""Benchmark: sparse-gate terms/s and the HBM / FP64 roofline fraction.

Workload (default, --workload mix60): the n=60 random-mix peaked circuit --
400 gates drawn uniformly from H, CNOT, CZ, RZ(theta ~ U[0, 2 pi)), Toffoli,
C3X and Haar-random U(8) on random qubits, the mirror with every inverse
perturbed as U^dagger exp(-i theta G) (theta ~ N(0, 0.05)), X on a seeded
hidden string -- with truncation to K = 2^26 terms and p = 0.9999 retained
mass after every gate, complex128 amplitudes.

One step = apply the next gate + truncate + read the peak (pipelined), on
the state once it has reached K terms: the whole hot path (key transform,
grouping, group mat-vec with zero drop, exact mass + select, renormalising
compaction, argmax).  The circuit from |0> up to the first gate on a full
state is run untimed, then --warmup steps, then exactly --steps steps.

value    : sum of input terms over the timed steps / device time of those
           steps (CUDA events on the library's stream; the state is resident
           in HBM and larger than L2, so no flush is needed).
e2e      : the same metric for the whole circuit run through the C ABI from
           the host (create, every gate with its matrix copied from pinned
           host memory, every truncation, the peak read back), wall clock.
roofline : the dominant kernel phase's algorithmic bytes (or FP64 flops) per
           launch over its CUDA-event launch time, against
           MEASURED_PEAKS.json (HBM) or the FP64 pipe.
c64      : the complex64 form on the same steps, and the error of the whole
           circuit's complex64 result against the complex128 result (which
           equals the CPU oracle bit for bit in every parity test).

--impl reference times the CPU oracle (test infrastructure; the only
reference that exists for this paper) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SM_COUNT, FP64_FMA_PER_SM_CLK = 148, 2      # B300 FP64 pipe: 2 DFMA / SM / clock (derived peak)
WORKLOADS = {
    "mix60": {"n": 60, "K": 1 << 26, "p": 0.9999, "seed": 1003,
              "desc": "n60 random mix (H, CNOT, CZ, RZ, Toffoli, C3X, Haar U(8)) x400 + perturbed mirror "
                      "(sigma 0.05) + X^s; top-K 2^26 and p=0.9999 after every gate"},
    "brick40": {"n": 40, "K": 1 << 24, "p": 1.0, "seed": 1002,
                "desc": "n40 brickwork Haar-SU(4) x8 + perturbed mirror + X^s, top-K 2^24 per gate, p=1"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mix60", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="c128", choices=["c128", "c64"])
    ap.add_argument("--K", type=int, default=0, help="override the workload's K")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-c64", action="store_true")
    ap.add_argument("--no-whole", action="store_true", help="skip the whole-circuit legs and the c64 error report")
    ap.add_argument("--no-ring", action="store_true", help="skip the ring u3/cz (fusion) leg")
    ap.add_argument("--no-ab", action="store_true", help="skip the group-first / expand-first comparison")
    ap.add_argument("--no-reserve", action="store_true",
                    help="let the buffers grow on demand instead of sizing them for K up front (profiling "
                         "runs: the device then holds about what the state needs)")
    ap.add_argument("--batch-circuits", type=int, default=512,
                    help="circuits of the batched-form leg (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the serving stream measured (0: skip the serving leg)")
    ap.add_argument("--requests-log", default="",
                    help="write one JSON line per request of the batched and serving legs to "
                         "<prefix>_batched.jsonl / <prefix>_serving.jsonl")
    a = ap.parse_args()
    w = dict(WORKLOADS[a.workload])
    if a.K:
        w["K"] = a.K
    a.wl = w
    return a


def make_circuit(wl, rank=0):
    from paper_2607_07816_b300 import circuits as C
    if wl["n"] == 60:
        return C.mix_n60(seed=wl["seed"] + rank, K=wl["K"], p=wl["p"])
    return C.brickwork_n40(seed=wl["seed"] + rank, layers=8, K=wl["K"], p=wl["p"])


def gate_kind(u) -> str:
    """diag / mono (one nonzero per row and column) / dense, from U's zero
    pattern (the library decides the same way)."""
    import numpy as np
    nz = np.abs(u) > 0
    if not (nz & ~np.eye(len(u), dtype=bool)).any():
        return "diag"
    if (nz.sum(0) == 1).all() and (nz.sum(1) == 1).all():
        return "mono"
    return "dense"


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
        self.path = os.path.join("/tmp", f"sv_clocks_{os.getpid()}_{device_index}.csv")

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


# ------------------------------------------------------------------ byte / flop model
def new_totals():
    keys = ["n_in", "n_pre", "n_kept", "steps", "select_levels", "selects", "window_hits", "window_terms",
            "sort_bytes", "heads_bytes", "apply_bytes", "compact_bytes", "window_bytes", "fp64_apply",
            "gates_diag", "gates_mono", "gates_dense", "cuts", "B_method", "B_strict"]
    return {k: 0 for k in keys}


def account_step(tot, q, kind, s1, s2, prec, n_bits):
    """Algorithmic bytes and FP64 work of one gate + truncation, per phase.
    Per term: key 8 B, probability 8 B, amplitude S_a (16 complex128, 8
    complex64); the grouping keeps a 4-byte index beside each key when
    n + log2 N exceeds 64 bits."""
    sa = 16 if prec == "c128" else 8
    S = 8 + sa
    m = len(q)
    n_in, n_pre, n_kept = s1["n_in"], s1["n_pre"], s2["n_kept"]
    pairs = 4 if n_bits + max(1, (max(1, n_in) - 1).bit_length()) > 64 else 0
    tot["n_in"] += n_in
    tot["n_pre"] += n_pre
    tot["n_kept"] += n_kept
    tot["steps"] += 1
    tot["select_levels"] += s2["select_levels"]
    tot["selects"] += s2["selects"]
    tot["window_hits"] += s2["window_hits"]
    tot["window_terms"] += s2["window_terms"]
    tot["gates_" + kind] += 1
    if kind != "diag":
        # count pass (8), scatter (read 8, write 8 + index), m merge levels (read + write)
        tot["sort_bytes"] += n_in * (8 + 16 + pairs) + m * n_in * (16 + 2 * pairs)
    if kind == "dense":
        tot["heads_bytes"] += 8 * n_in
    if kind == "diag":
        tot["apply_bytes"] += n_in * (8 + sa) + n_in * (sa + 8)
    else:  # grouped key (+ index) and gathered amplitude per input; key, amplitude, probability per output
        tot["apply_bytes"] += n_in * (8 + pairs + sa) + n_pre * (16 + sa)
    # FP64 pipe operations of the apply kernel, 2 flops each: complex128 runs
    # 4 fused multiply-adds per (input, output) pair with a nonzero entry;
    # every candidate's probability is a multiply + fma in FP64
    ops = 2.0 * n_pre
    if prec == "c128":
        ops += 4.0 * n_in * ((1 << m) if kind == "dense" else 1)
    tot["fp64_apply"] += 2.0 * ops
    tot["window_bytes"] += 8 * n_pre * s2["selects"]
    cut = n_kept < n_pre
    if cut:
        tot["cuts"] += 1
        # keep flags, the kept terms' keys and amplitudes read and written
        # (the compaction writes no probabilities)
        tot["compact_bytes"] += n_pre / 8 + 2 * (8 + sa) * n_kept
    # gate-level byte model B_method: group 2 S N_in, mat-vec S (N_in + N_pre),
    # select 8 N_pre and compaction S (N_pre + N_kept) when a cut is made
    b = 2 * S * n_in + S * (n_in + n_pre)
    if cut:
        b += 8 * n_pre + S * (n_pre + n_kept)
    tot["B_method"] += b
    tot["B_strict"] += S * (n_in + n_kept)


def phase_bytes(ph, tot):
    return {"sort": tot["sort_bytes"], "heads": tot["heads_bytes"], "apply": tot["apply_bytes"],
            "window": tot["window_bytes"], "select": 16 * tot["window_terms"],
            "compact": tot["compact_bytes"], "peak": 16 * 1184 * tot["steps"]}.get(ph, 0.0)


def attainable_ms(tot, bw_gbs, fp64_tflops):
    """The steps' time if every phase ran at its own roof: the larger of its
    algorithmic bytes over the HBM bandwidth and its FP64 work over the
    measured FP64 rate (the gate's mat-vec; the compaction's rescale: 2 FP64
    multiplies per kept term), summed over the phases."""
    bw, f = bw_gbs * 1e9, fp64_tflops * 1e12
    t = max(tot["apply_bytes"] / bw, tot["fp64_apply"] / f)
    t += max(tot["compact_bytes"] / bw, 4.0 * tot["n_kept"] / f)
    t += (tot["sort_bytes"] + tot["heads_bytes"] + tot["window_bytes"] + 16 * tot["window_terms"]) / bw
    return 1e3 * t


def fp64_derived_tflops(sm_mhz):
    return SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12


def roofline(res, prec, peaks, fp64_probe):
    # the phase times come from the instrumented steps: their own gates' totals
    tot, phases = res["phase_totals"], res["phases"]
    dom = max((p for p in phases if p != "other"), key=lambda p: phases[p][0])
    ms, launches = phases[dom]
    per_launch_s = ms / 1e3 / max(1, launches)
    bytes_per_launch = phase_bytes(dom, tot) / max(1, launches)
    gbs = bytes_per_launch / per_launch_s / 1e9
    hbm_frac = gbs / peaks["hbm_gbs"]
    out = {"kernel": dom, "bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": round(hbm_frac, 4), "traffic": traffic_for(dom, prec, bytes_per_launch),
           "peak_src": f"{peaks['src']} copy bandwidth (MEASURED_PEAKS.json)",
           "launch_ms": round(per_launch_s * 1e3, 4), "launches": launches,
           "alg_bytes_per_launch": round(bytes_per_launch)}
    if dom == "apply" and tot["fp64_apply"] > 0:
        fp64_peak = fp64_derived_tflops(peaks["sm_max_mhz"])
        tflops = tot["fp64_apply"] / max(1, launches) / per_launch_s / 1e12
        if tflops / fp64_peak > hbm_frac:
            out.update({"bound": "alu", "achieved": round(tflops, 4), "peak": round(fp64_peak, 4),
                        "unit": "TFLOP/s", "frac": round(tflops / fp64_peak, 4),
                        "peak_src": "FP64 pipe derived: 148 SMs x 2 DFMA/clk x 2 flop x max SM clock",
                        "fp64_probe_tflops": fp64_probe,
                        "frac_of_probe": round(tflops / fp64_probe, 4) if fp64_probe else None,
                        "hbm_frac": round(hbm_frac, 4)})
    return out


def traffic_for(phase, prec, alg_bytes):
    """DRAM bytes per launch of the phase's dominant kernel from the
    committed ncu summary, when it was taken on the current kernel sources
    (else null)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        from paper_2607_07816_b300 import build as B
        if d.get("source_hash") != B.source_hash():
            return None
        ent = d["kernels"].get(f"{phase}/{prec}")
        if not ent:
            return None
        return round(ent["dram_bytes_per_alg_byte"] * alg_bytes)
    except Exception:
        return None


# ------------------------------------------------------------------ our arm
def run_steps(args, rank, prec_name, dev, stream, sample_clocks):
    """The timed steps on the state at K terms, then as many instrumented
    steps for the per-phase breakdown."""
    import torch
    from paper_2607_07816_b300 import sv
    wl = args.wl
    prec = sv.SV_C128 if prec_name == "c128" else sv.SV_C64
    circ = make_circuit(wl, rank)
    gates = circ.gates
    kinds = [gate_kind(u) for _, u in gates]
    st = sv.SparseState(circ.n, wl["K"], wl["p"], prec=prec, stream=stream.cuda_stream)
    if not args.no_reserve:
        st.reserve(wl["K"])  # every buffer sized for K-term states: no allocation inside the steps
    gi = 0
    # ramp: the circuit from |0> until the state is at K terms (the p-mass cut
    # may keep it slightly below K: 99% counts as full)
    while gi < len(gates) and st.num_terms() < 0.99 * wl["K"]:
        q, u = gates[gi]
        st.apply_gate(q, u)
        st.truncate()
        gi += 1
    first_full = gi
    for _ in range(args.warmup):
        q, u = gates[gi % len(gates)]
        st.apply_gate(q, u)
        st.truncate()
        st.peak()
        gi += 1
    torch.cuda.synchronize(dev)
    barrier()
    tot = new_totals()
    clocks = ClockSampler(dev.index) if sample_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    l0 = sv.sv_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    g_start = gi
    # checkpoint (untimed): the per-phase pass below replays the same gates
    ck_keys, ck_amps = st.export()
    torch.cuda.synchronize(dev)
    pending = None
    # an NVTX range names the timed steps (a profiler can select their launches)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        j = gi % len(gates)
        q, u = gates[j]
        gi += 1
        st.apply_gate(q, u)
        s1 = st.stats()
        st.truncate()
        # the peak of every step, read back pipelined: its 16 bytes reach the
        # host while the next step runs
        ticket = st.peak_async()
        s2 = st.stats()
        if pending is not None:
            st.peak_wait(pending)
        pending = ticket
        account_step(tot, q, kinds[j], s1, s2, prec_name, circ.n)
    if pending is not None:
        st.peak_wait(pending)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    launches = sv.sv_launch_count() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    barrier()
    rate, units_all, ms_all = whole_job_rate(tot["n_in"], ms)
    # per-phase breakdown: the same gates again from the checkpoint, with CUDA
    # events around each phase (events between the kernels of a step cost
    # time of their own, so they stay out of the timed loop)
    st.load(ck_keys, ck_amps)
    del ck_keys, ck_amps
    gi = g_start
    st.set_timing(True)
    ph_tot = new_totals()
    for _ in range(args.steps):
        j = gi % len(gates)
        q, u = gates[j]
        gi += 1
        st.apply_gate(q, u)
        s1 = st.stats()
        st.truncate()
        s2 = st.stats()
        st.peak_wait(st.peak_async())
        account_step(ph_tot, q, kinds[j], s1, s2, prec_name, circ.n)
    torch.cuda.synchronize(dev)
    phases = st.phase_times()
    fin = st.stats()
    st.close()
    phase_sum = sum(v[0] for v in phases.values())
    return {"ms": ms, "totals": tot, "phases": phases, "phase_totals": ph_tot, "launches": launches,
            "phase_sum_ms": phase_sum,
            "clocks": clk, "rate": rate, "units_all": units_all, "first_full_gate": first_full,
            "timed_gates": [g_start, g_start + args.steps - 1],
            "paths": {k: fin[k] for k in ("local_gates", "global_gates", "diag_gates", "mono_gates")}}


def run_whole(args, rank, prec_name, dev, stream):
    """The whole circuit from |0>, every gate truncated; CUDA-event time on
    the library's stream; the final state kept for the error report."""
    import torch
    from paper_2607_07816_b300 import sv
    wl = args.wl
    prec = sv.SV_C128 if prec_name == "c128" else sv.SV_C64
    circ = make_circuit(wl, rank)
    st = sv.SparseState(circ.n, wl["K"], wl["p"], prec=prec, stream=stream.cuda_stream)
    st.reserve(wl["K"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    n_in = n_pre = 0
    e0.record(stream)
    for (q, u) in circ.gates:
        st.apply_gate(q, u)
        s1 = st.stats()
        n_in += s1["n_in"]
        n_pre += s1["n_pre"]
        st.truncate()
    key, pr = st.peak()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    F = st.retained_mass()
    keys, amps = st.export()
    st.close()
    return {"ms": ms, "terms": n_in, "candidates": n_pre, "terms_per_s": n_in / (ms / 1e3),
            "gates": len(circ.gates), "peak_key": key, "peak_prob": pr, "peak_is_hidden": key == circ.hidden,
            "retained_mass": F, "final_terms": len(keys)}, (keys, amps)


def error_report(ref, test, dev):
    """complex64 final state against the complex128 one, on the GPU: max
    |d amp| on the common keys, the symmetric difference (count and its
    probability mass on the side that has it) and the L2 distance over the
    union (absent = 0)."""
    import numpy as np
    import torch
    k0, a0 = ref
    k1, a1 = test
    K0 = torch.from_numpy(k0.view(np.int64)).to(dev)
    K1 = torch.from_numpy(k1.view(np.int64)).to(dev)
    A0 = torch.from_numpy(np.ascontiguousarray(a0)).to(dev)
    A1 = torch.from_numpy(np.ascontiguousarray(a1.astype(np.complex128))).to(dev)
    s0, i0 = torch.sort(K0)
    s1, i1 = torch.sort(K1)
    pos = torch.searchsorted(s0, s1).clamp(max=len(s0) - 1)
    hit1 = s0[pos] == s1                     # test keys present in ref
    in0 = torch.zeros(len(s0), dtype=torch.bool, device=dev)
    in0[pos[hit1]] = True
    a0s, a1s = A0[i0], A1[i1]
    d = (a0s[pos[hit1]] - a1s[hit1]).abs()
    only0 = (a0s[~in0].abs() ** 2).sum().item()
    only1 = (a1s[~hit1].abs() ** 2).sum().item()
    l2 = float(np.sqrt((d ** 2).sum().item() + only0 + only1))
    out = {"terms_ref": len(k0), "terms": len(k1), "common": int(hit1.sum().item()),
           "max_abs_amp_err_common": float(d.max().item()) if d.numel() else 0.0,
           "sym_diff_count": int((~in0).sum().item() + (~hit1).sum().item()),
           "sym_diff_mass": only0 + only1, "union_l2": l2}
    del K0, K1, A0, A1, s0, s1, i0, i1, pos, hit1, in0, a0s, a1s, d
    torch.cuda.empty_cache()
    return out


def run_e2e(args, rank, dev, stream):
    import numpy as np
    import torch
    from paper_2607_07816_b300 import sv
    wl = args.wl
    circ = make_circuit(wl, rank)
    prec = sv.SV_C128 if args.prec == "c128" else sv.SV_C64
    # host-resident inputs: the gate matrices in pinned host memory
    pinned = [(q, torch.from_numpy(np.ascontiguousarray(u)).pin_memory().numpy()) for (q, u) in circ.gates]
    torch.cuda.synchronize(dev)
    barrier()
    h0, d0 = sv.sv_transfer_bytes()
    t0 = time.perf_counter()
    st = sv.SparseState(circ.n, wl["K"], wl["p"], prec=prec, stream=stream.cuda_stream)
    st.reserve(wl["K"])  # part of the timed region: the allocation a user's run pays once
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
            "scope": "whole circuit from |0> (every gate a step), host wall clock",
            "peak_is_hidden": bool(key == circ.hidden), "peak_prob": pr}


AMP_TOL_C64 = 2e-6  # amplitude error allowed to the complex64 form on a peaked request


def is_peaked(s) -> bool:
    """A request's complex128 final state has a clear top: the top
    probability exceeds the runner-up by more than the complex64 error
    allows (relative gap > 1e-3) and the retained mass is above 1e-6."""
    return s["gap"] > 1e-3 and s["F"] > 1e-6


def amp_error(keys_a, amps_a, keys_b, amps_b):
    """max |a - b| over the keys both states hold, and the count and
    probability mass (in b) of the keys only one of them holds."""
    import numpy as np
    common, ia, ib = np.intersect1d(keys_a, keys_b, assume_unique=True, return_indices=True)
    err = float(np.max(np.abs(amps_a[ia].astype(np.complex128) - amps_b[ib]))) if len(common) else 0.0
    only_b = np.ones(len(keys_b), dtype=bool)
    only_b[ib] = False
    return err, len(keys_a) + len(keys_b) - 2 * len(common), float(np.sum(np.abs(amps_b[only_b]) ** 2))


def peaked_check(batched, serial, circuits, checked=None):
    """Peaks of the complex64 batched results against the serial complex128
    results, over all requests and over the peaked ones (is_peaked).  With
    `checked` (complex64 results holding the final states of the peaked
    requests) the amplitudes of every peaked request are compared with the
    complex128 state on the common keys as well."""
    peaked = same = 0
    diff_peaked = []
    errs = []
    for j, (b, s) in enumerate(zip(batched, serial)):
        if is_peaked(s):
            peaked += 1
            if b.peak_key == s["key"]:
                same += 1
            else:
                diff_peaked.append(j)
            if checked is not None and checked[j] is not None and checked[j].keys is not None and "keys" in s:
                errs.append((j,) + amp_error(checked[j].keys, checked[j].amps, s["keys"], s["amps"]))
    all_same = sum(int(b.peak_key == s["key"]) for b, s in zip(batched, serial))
    out = {"identical_peaks_all": f"{all_same}/{len(serial)}",
           "peaked_requests": peaked, "identical_peaks_on_peaked": f"{same}/{peaked}",
           "peaked_rule": "complex128 top-two relative probability gap > 1e-3 and retained mass > 1e-6",
           "differing_peaked_indices": diff_peaked[:20]}
    if errs:
        def part(rows):
            if not rows:
                return {"requests": 0}
            e = [x[1] for x in rows]
            over = [x[0] for x in rows if x[1] > AMP_TOL_C64]
            return {"requests": len(rows), "max_abs_amp_err": max(e), "median_abs_amp_err": statistics.median(e),
                    "within_tol": f"{len(rows) - len(over)}/{len(rows)}", "over_tol_indices": over[:20],
                    "max_sym_diff_count": max(x[2] for x in rows), "max_sym_diff_mass": max(x[3] for x in rows)}
        # where both precisions kept the same terms the difference is the
        # arithmetic's; where the truncations kept different sets (a cut
        # among probabilities closer than float32 resolves), it is the set's
        out["amp_check_on_peaked"] = {
            "tol": AMP_TOL_C64,
            "same_kept_set": part([x for x in errs if x[2] == 0]),
            "different_kept_set": part([x for x in errs if x[2] != 0]),
            "scope": "complex64 batched final state vs complex128 serial: max |a64 - a128| over the keys both "
                     "hold; sym_diff = keys held by one of them only (count, complex128 mass)"}
    return out


def request_table(circuits, batched, serial):
    """Per request: size, the complex64 batched result (peak probability,
    retained mass) and the complex128 serial one."""
    rows = []
    for j, (c, b, s) in enumerate(zip(circuits, batched, serial)):
        rows.append({"j": j, "n": c.n, "K": c.K, "gates": len(c.gates), "peaked": is_peaked(s),
                     "c64_peak_prob": b.peak_prob, "c64_retained_mass": b.retained_mass,
                     "c128_peak_prob": s["prob"], "c128_retained_mass": s["F"],
                     "same_peak": bool(b.peak_key == s["key"])})
    return rows


def quantiles(v):
    import numpy as np
    v = np.asarray(v, dtype=float)
    return {"min": float(v.min()), "p50": float(np.median(v)), "max": float(v.max())} if len(v) else None


def request_summary(rows, path=None):
    if path:
        with open(path, "w") as f:
            for r in rows:
                f.write(json.dumps(r) + "\n")
    return {"c64_retained_mass": quantiles([r["c64_retained_mass"] for r in rows]),
            "c64_peak_prob": quantiles([r["c64_peak_prob"] for r in rows]),
            "c64_peak_prob_on_peaked": quantiles([r["c64_peak_prob"] for r in rows if r["peaked"]]),
            "log": path}


def serial_c128(circuits, stream, arrivals=None, keep_peaked=False):
    """The serial plain path: every circuit alone on the single-state
    complex128 API, one after the other (waiting for each arrival when
    arrival times are given); per circuit: service time, finish time, peak,
    runner-up gap and retained mass (with keep_peaked, also the final state
    of every peaked request, read off the clock)."""
    from paper_2607_07816_b300 import sv
    out = []
    t0 = time.perf_counter()
    for j, c in enumerate(circuits):
        if arrivals is not None:
            wait = arrivals[j] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        ts = time.perf_counter()
        st = sv.SparseState(c.n, c.K, 1.0, prec=sv.SV_C128, stream=stream)
        for (q, u) in c.gates:
            st.apply_gate(q, u)
            st.truncate()
        key, prob = st.peak()
        te = time.perf_counter()
        # the runner-up (canonical dump) for the peakedness rule: not part of
        # the service, so its time is taken off the clock
        _, probs = st.probs()
        F = st.retained_mass()
        second = float(probs[1]) if len(probs) > 1 else 0.0
        rec = {"key": key, "prob": prob, "F": F, "gap": (prob - second) / prob if prob > 0 else 0.0}
        if keep_peaked and is_peaked(rec):
            rec["keys"], rec["amps"] = st.export()
        st.close()
        t0 += time.perf_counter() - te
        rec.update({"svc": te - ts, "finish": te - t0})
        out.append(rec)
    return out


def peaked_states_c64(circuits, serial, n_max, stream):
    """The complex64 batched final states of the peaked requests (an
    untimed run of the same serving loop)."""
    from paper_2607_07816_b300 import serve, sv
    want = [j for j, s in enumerate(serial) if is_peaked(s)]
    srv = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=stream)
    try:
        return srv.run(circuits, export=want)
    finally:
        srv.close()


def run_batched(args, rank, dev, stream):
    """Config-4 leg: the seeded batch of mirrored brickwork circuits (n in
    [16,48], depth in [2,10], K = 2^k with k in [10,20]) all present at t=0,
    on the complex64 batched serving loop, against the serial complex128
    plain path on the same GPU (measured)."""
    import torch
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300 import serve, sv
    R = args.batch_circuits
    circs = C.batch_circuits(R)
    n_max = max(c.n for c in circs)
    s = stream.cuda_stream
    warm = [c for c in circs if c.K <= 1 << 12][:4]
    serial_c128(warm, s)
    for one_launch in (True, False):
        w = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=s, one_launch=one_launch)
        w.run(warm)
        w.close()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ser = serial_c128(circs, s, keep_peaked=True)  # the peaked states are read off the clock
    serial_s = time.perf_counter() - t0
    # the step as one persistent launch (the default) and as separate kernels
    forms, res = {}, None
    for name, one_launch in (("one_launch", True), ("kernels", False)):
        srv = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=s, one_launch=one_launch)
        t0 = time.perf_counter()
        got = srv.run(circs)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        forms[name] = {"circuits_per_s": R / wall, "wall_s": wall, "steps": srv.steps,
                       "graphs": srv.batch.graph_stats()}
        if one_launch:
            forms[name]["phases_ms"] = {k: round(v, 2) for k, v in srv.batch.layer_phase_times().items()}
            res = got
        else:
            forms[name]["results_equal_to_one_launch"] = "%d/%d" % (
                sum(int((a.peak_key, a.peak_prob, a.retained_mass) == (b.peak_key, b.peak_prob, b.retained_mass))
                    for a, b in zip(res, got)), R)
        srv.close()
    batched_s = forms["one_launch"]["wall_s"]
    out = {"circuits": R, "prec": "c64 batched vs c128 serial", "serial_circuits_per_s": R / serial_s,
           "batched_circuits_per_s": R / batched_s, "speedup": serial_s / batched_s,
           "form": "one persistent launch per step (graph replay, no host wait)",
           "steps": forms["one_launch"]["steps"], "serial_s": serial_s, "batched_s": batched_s, "forms": forms,
           "kernels_speedup": serial_s / forms["kernels"]["wall_s"]}
    out.update(peaked_check(res, ser, circs, peaked_states_c64(circs, ser, n_max, s)))
    log = args.requests_log + "_batched.jsonl" if args.requests_log else None
    out["per_request"] = request_summary(request_table(circs, res, ser), log)
    return out


def run_serving(args, rank, dev, stream):
    """Config-5 leg (first R requests of the seeded serving stream: mirrored
    brickwork circuits as in config 4 plus a 2% share of large ones, n=56,
    depth 12, K=2^25).  batched_closed: the continuous-batching loop
    (complex64, 160 GB budget) with all requests at t=0 gives the capacity;
    served: Poisson arrivals at 80% of it, arrival-to-peak latency; serial:
    the single-state complex128 path serving the same arrival stream one
    request at a time (measured, waiting for each arrival)."""
    import numpy as np
    import torch
    from paper_2607_07816_b300 import circuits as C
    from paper_2607_07816_b300 import serve, sv
    R = args.serve_requests
    reqs = [C.serving_request(j) for j in range(R)]
    n_max = max(c.n for c in reqs)
    s = stream.cuda_stream
    torch.cuda.synchronize(dev)
    srv = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=s)
    t0 = time.perf_counter()
    closed = srv.run(reqs)
    torch.cuda.synchronize(dev)
    closed_s = time.perf_counter() - t0
    steps_closed, resident = srv.steps, srv.peak_resident
    srv.close()
    capacity = R / closed_s
    rate = 0.8 * capacity
    arrivals = serve.poisson_arrivals(R, rate, 1005)
    srv = serve.Server(160 << 30, n_max=n_max, prec=sv.SV_C64, stream=s)
    t0 = time.perf_counter()
    opened = srv.run(reqs, arrivals=arrivals)
    torch.cuda.synchronize(dev)
    open_s = time.perf_counter() - t0
    srv.close()
    p50, p99 = serve.percentiles(opened)
    ser = serial_c128(reqs, s, arrivals=arrivals, keep_peaked=True)
    s_lat = np.array([x["finish"] - a for x, a in zip(ser, arrivals)])
    serial_cps = R / sum(x["svc"] for x in ser)
    out = {"requests": R, "large_requests": sum(int(c.n == 56) for c in reqs), "budget_gb": 160,
           "batched_closed": {"circuits_per_s": capacity, "wall_s": closed_s, "steps": steps_closed,
                              "max_resident": resident},
           "served": {"arrival_rate": rate, "circuits_per_s": R / (max(r.finished for r in opened) - arrivals[0]),
                      "p50_s": p50, "p99_s": p99, "wall_s": open_s},
           "serial_measured": {"circuits_per_s": serial_cps, "p50_s": float(np.percentile(s_lat, 50)),
                               "p99_s": float(np.percentile(s_lat, 99)),
                               "note": "the same arrival stream served one request at a time (queue grows: "
                                       "arrivals exceed the serial capacity)"},
           "speedup_circuits_per_s": capacity / serial_cps,
           "served_results_equal_to_saturated_run": "%d/%d" % (
               sum(int(a.peak_key == b.peak_key and a.peak_prob == b.peak_prob) for a, b in zip(opened, closed)), R)}
    out.update(peaked_check(closed, ser, reqs, peaked_states_c64(reqs, ser, n_max, s)))
    log = args.requests_log + "_serving.jsonl" if args.requests_log else None
    out["per_request"] = request_summary(request_table(reqs, closed, ser), log)
    return out


def run_variant_ab(args, rank, dev, stream, steps=8):
    """Group-first (default: grouping by partition and merge) against
    group-first with a full radix sort and against expand-first (the paper's
    formulation: one record per term and output, sorted, then summed per
    output) on the n=40 brickwork state at 2^24 terms: the same gates,
    alternating blocks of steps, CUDA-event time per step on the library's
    stream."""
    import torch
    from paper_2607_07816_b300 import sv
    wl = WORKLOADS["brick40"]
    circ = make_circuit(wl, rank)
    st = sv.SparseState(circ.n, wl["K"], 1.0, prec=sv.SV_C128, stream=stream.cuda_stream)
    gi = 0
    while gi < len(circ.gates) and st.num_terms() < wl["K"]:
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
    return {"workload": "n40 brickwork at K=2^24", "steps_each": steps, "group_first_ms_per_step": round(g, 3),
            "group_first_radix_sort_ms_per_step": round(r, 3),
            "expand_first_ms_per_step": round(e, 3), "expand_over_group": round(e / g, 3),
            "radix_over_merge_grouping": round(r / g, 3)}


def run_ring(args, dev, stream):
    """The ring-connected u3/cz workload shaped like the paper's example (44
    qubits, 93 (u3, u3, cz) blocks walking the ring, their perturbed mirror,
    X on a seeded hidden string: about 580 instructions), whole, as given,
    after reordering and fusion into 2-qubit blocks, and fused into blocks of
    up to 4 qubits: updates, wall time, and whether the peak is the hidden
    string."""
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


def run_ours(args, rank, world):
    import torch
    from paper_2607_07816_b300 import sv
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sv.load_library()
    res = {"main": run_steps(args, rank, args.prec, dev, stream, sample_clocks=True)}
    res["fp64_probe_tflops"] = round(sv.sv_probe_fp64(1 << 14, 4)[0], 4)
    if not args.no_c64 and args.prec == "c128":
        res["c64"] = run_steps(args, rank, "c64", dev, stream, sample_clocks=False)
    if not args.no_whole:
        w128, f128 = run_whole(args, rank, "c128", dev, stream)
        res["whole"] = {"c128": w128}
        if not args.no_c64:
            w64, f64 = run_whole(args, rank, "c64", dev, stream)
            res["whole"]["c64"] = w64
            res["whole"]["c64_vs_c128"] = error_report(f128, f64, dev)
            res["whole"]["c64_vs_c128"]["peak_identical"] = w64["peak_key"] == w128["peak_key"]
            del f64
        del f128
    if not args.no_e2e:
        res["e2e"] = run_e2e(args, rank, dev, stream)
    if args.batch_circuits > 0:
        res["batched"] = run_batched(args, rank, dev, stream)
    if args.serve_requests > 0:
        res["serving"] = run_serving(args, rank, dev, stream)
    if not args.no_ring:
        res["ring"] = run_ring(args, dev, stream)
    if not args.no_ab:
        res["variant_ab"] = run_variant_ab(args, rank, dev, stream)
    return res


# ------------------------------------------------------------------ CPU / reference arm
def oracle_sample(wl, seconds: float, max_gates: int = 10 ** 9):
    """The oracle as it stands, single-threaded, on the same circuit and K
    from |0...0>, gate after gate until `seconds` of CPU work have elapsed
    (the first gates: the state has not reached K within the sample)."""
    import oracle
    circ = make_circuit(wl)
    o = oracle.Oracle(circ.n, wl["K"], wl["p"])
    n_in, g = 0, 0
    t0 = time.perf_counter()
    last = 0.0
    while g < min(len(circ.gates), max_gates):
        # stop before a gate that would overrun the budget (a gate can
        # multiply the term count by up to 16)
        if g > 0 and time.perf_counter() - t0 + 8 * last > seconds:
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
            "sample": f"{wl['desc']}: gates 1..{g} from |0> ({n_in} input terms, largest state "
                      f"{o.num_terms()} terms) in {dt:.1f} s, single-threaded C++ std::map oracle"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle  # noqa: F401  (builds the oracle if needed)
    wl = args.wl
    per = []
    for i in range(args.warmup + args.steps):
        s = oracle_sample(wl, seconds=1.0)
        if i >= args.warmup:
            per.append(s)
    v = statistics.mean(p["value"] for p in per)
    line = {"metric": "sparse-gate terms/s", "value": v, "unit": "terms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_of(args, world),
            "cpu_baseline": {"value": v, "unit": "terms/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: " + per[0]["sample"]},
            "e2e": {"value": v, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def config_of(args, world):
    wl = args.wl
    return {"workload": wl["desc"], "n": wl["n"], "K": wl["K"], "p": wl["p"], "prec": args.prec,
            "seed": wl["seed"], "l2": "state larger than L2 (no flush needed)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


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
    peaks = measured_peaks()
    res = run_ours(args, rank, world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    m = res["main"]
    tot = m["totals"]
    ms = m["ms"]
    bw = peaks["hbm_gbs"] * 1e9
    line = {
        "metric": "sparse-gate terms/s", "value": m["rate"], "unit": "terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.prec == "c128" else "f32",
        "data": "synthetic (seeded random-mix mirror circuit)" if args.wl["n"] == 60
        else "synthetic (seeded Haar brickwork mirror circuit)",
        "config": config_of(args, world),
        "roofline": roofline(m, args.prec, peaks, res["fp64_probe_tflops"]),
        "gate_roofline": {"B_method_frac": round(tot["B_method"] / (ms / 1e3) / bw, 4),
                          "B_strict_frac": round(tot["B_strict"] / (ms / 1e3) / bw, 4),
                          "peak_gbs": peaks["hbm_gbs"],
                          "attainable_ms": round(attainable_ms(tot, peaks["hbm_gbs"], res["fp64_probe_tflops"]), 3),
                          "frac_of_attainable": round(attainable_ms(tot, peaks["hbm_gbs"], res["fp64_probe_tflops"]) / ms, 4),
                          "B_method_frac_at_attainable": round(
                              tot["B_method"] / (attainable_ms(tot, peaks["hbm_gbs"], res["fp64_probe_tflops"]) / 1e3) / bw, 4),
                          "note": "attainable: each phase at the larger of bytes / HBM and FP64 work / the FP64 probe"},
        "phases_ms": {k: round(v[0], 3) for k, v in m["phases"].items()},
        "phase_launches": {k: v[1] for k, v in m["phases"].items()},
        "phases_note": "the timed steps' gates replayed from a checkpoint with CUDA events around each phase; "
                       "the timed loop minus the phase sum is host orchestration and launch gaps",
        "phase_sum_ms": round(m["phase_sum_ms"], 3),
        "gpu_launches": m["launches"],
        "clocks": m["clocks"],
        "fp64_probe_tflops": res["fp64_probe_tflops"],
        "timed_gates": m["timed_gates"], "first_full_gate": m["first_full_gate"],
        "totals": {k: (round(v) if isinstance(v, float) else v) for k, v in tot.items()},
        "gate_paths": m["paths"],
    }
    if "c64" in res:
        c = res["c64"]
        ct = c["totals"]
        line["c64"] = {"value": c["rate"], "unit": "terms/s", "ms_per_step": c["ms"] / args.steps,
                       "B_method_frac": round(ct["B_method"] / (c["ms"] / 1e3) / bw, 4),
                       "frac_of_attainable": round(attainable_ms(ct, peaks["hbm_gbs"], res["fp64_probe_tflops"])
                                                   / c["ms"], 4),
                       "roofline": roofline(c, "c64", peaks, res["fp64_probe_tflops"]),
                       "phases_ms": {k: round(v[0], 3) for k, v in c["phases"].items()}}
    if "whole" in res:
        line["whole_circuit"] = res["whole"]
        if "c64" in line and "c64_vs_c128" in res["whole"]:
            line["c64"]["error_vs_c128_whole_circuit"] = res["whole"]["c64_vs_c128"]
    for key, name in (("e2e", "e2e"), ("batched", "batched"), ("serving", "serving"), ("ring", "ring_u3cz"),
                      ("variant_ab", "apply_variant_ab")):
        if key in res:
            line[name] = res[key]
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = oracle_sample(args.wl, seconds=15.0)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
