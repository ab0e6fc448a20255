#!/usr/bin/env python
"""Throughput of the compressed streamed state-vector path on GB300.

Default workload (the configuration the headline metric is quoted on):
n = 30 qubits, complex64, chunks of 2^22 amplitudes held compressed in pinned
host memory (error bound 1e-6), a depth-40 random layered circuit (H / RX / RZ
on every qubit, then a CNOT on a seeded random pairing per layer; 1800
gates), streamed through the GPU in groups of 2^g chunks (g chosen by the
library from the free device memory: 6 here, four groups per pass). One step = one
sv_apply_circuit of that circuit: every pass streams all chunks host -> GPU,
decodes, applies the fused gates in on-chip tiles, re-encodes (with the FP64
norm) and streams them back.

Metric: amplitude-gate updates per second = gates * 2^n / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload {layers30,ghz30,qft30,qft16,layers16,
                              ghz36,qft36,clifford36,grad-hea24,grad-hea32,grad-hea32-ckpt1,
                              grad-hea28,qft36-rel,clifford36-rel,layers30-rel}
  (-rel: the relative error bound, each chunk's step from its largest component)

With --gpus N under torchrun every rank runs an independent replica of the
workload (weak scaling, no data-path collective); rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "amp-gate updates/s"

# name -> (n, chunk qubits, eb, dtype, group qubits, circuit, extra)
WORKLOADS = {
    "layers30": dict(n=30, c=22, eb=1e-6, dtype="c64", group=0, circuit="layers", depth=40),
    "ghz30": dict(n=30, c=22, eb=1e-6, dtype="c64", group=0, circuit="ghz"),
    "qft30": dict(n=30, c=22, eb=1e-6, dtype="c64", group=0, circuit="qft"),
    "qft16": dict(n=16, c=10, eb=1e-6, dtype="c128", group=0, circuit="qft"),
    "layers16": dict(n=16, c=10, eb=1e-6, dtype="c128", group=0, circuit="layers", depth=20),
    "ghz36": dict(n=36, c=26, eb=1e-5, dtype="c64", group=0, circuit="ghz"),
    "qft36": dict(n=36, c=26, eb=1e-5, dtype="c64", group=0, circuit="qft"),
    "clifford36": dict(n=36, c=26, eb=1e-5, dtype="c64", group=0, circuit="clifford", depth=30),
    # the same with the relative error bound (step from each chunk's largest component)
    # n = 36 under the relative bound at the tightest eb whose store fits 70 % of the GPU machine's host
    # memory (at 1e-5 a spread 36-qubit state needs ~300 GB per copy)
    "qft36-rel": dict(n=36, c=26, eb=2.0 ** -5, dtype="c64", group=0, circuit="qft", relative=True),
    "clifford36-rel": dict(n=36, c=26, eb=2.0 ** -5, dtype="c64", group=0, circuit="clifford", depth=30,
                            relative=True),
    "layers30-rel": dict(n=30, c=22, eb=1e-6, dtype="c64", group=0, circuit="layers", depth=40, relative=True),
    "grad-hea24": dict(n=24, c=24, eb=0.0, dtype="c64", group=0, circuit="hea", layers=10, mode="uncompressed"),
    "grad-hea32": dict(n=32, c=24, eb=1e-6, dtype="c64", group=0, circuit="hea", layers=8, sets=16),
    # the same with psi checkpointed after every forward pass (checkpoint_passes = 1)
    "grad-hea32-ckpt1": dict(n=32, c=24, eb=1e-6, dtype="c64", group=0, circuit="hea", layers=8, sets=16,
                             checkpoint=1),
    # a small compressed gradient with config 4's chunks (16 chunks of 2^24): profiling case
    "grad-hea28": dict(n=28, c=24, eb=1e-6, dtype="c64", group=0, circuit="hea", layers=2),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="layers30", choices=sorted(WORKLOADS))
    p.add_argument("--eb", type=float, default=None)
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--chunk", type=int, default=None)
    p.add_argument("--depth", type=int, default=None)
    p.add_argument("--group", type=int, default=None)
    p.add_argument("--sets", type=int, default=None, help="parameter sets for grad-hea32")
    p.add_argument("--no-extras", action="store_true", help="skip the comparator and baseline legs")
    p.add_argument("--table1", action="store_true",
                   help="the paper's Table 1: host<->device copy strategies at 20 and 25 qubits")
    p.add_argument("--jit", type=int, default=1, choices=[0, 1],
                   help="1: sub-pass kernels generated per gate sequence (default); 0: table-driven kernel")
    p.add_argument("--remap", action="store_true",
                   help="sv_config.remap_qubits: move qubits between chunk-index and in-chunk positions "
                        "when that saves passes")
    a = p.parse_args()
    w = dict(WORKLOADS[a.workload])
    for k, v in (("eb", a.eb), ("n", a.n), ("c", a.chunk), ("depth", a.depth), ("group", a.group),
                 ("sets", a.sets)):
        if v is not None:
            w[k] = v
    if w["c"] > w["n"]:
        w["c"] = w["n"]
    a.w = w
    return a


def make_circuit(w, seed=1):
    n = w["n"]
    if w["circuit"] == "layers":
        return W.random_layers(n, w["depth"], seed=seed)
    if w["circuit"] == "ghz":
        return W.ghz(n)
    if w["circuit"] == "qft":
        return W.qft(n)
    if w["circuit"] == "clifford":
        return W.random_clifford_rz(n, w["depth"], 10, seed=seed)
    raise ValueError(w["circuit"])


def host_budget():
    """Pinned host memory the library may take: 70 % of the host's memory
    (it then fails with SV_ERR_HOST_OOM instead of exhausting the host)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemTotal:"):
                    return int(0.7 * int(line.split()[1]) * 1024)
    except OSError:
        pass
    return 0


def describe(w, ngates, group=None):
    if w["circuit"] == "hea":
        return (f"adjoint gradient, hardware-efficient ansatz n={w['n']}, {w['layers']} layers, 1-D Ising, "
                f"{w['dtype']}, " + ("uncompressed in HBM" if w.get("mode") == "uncompressed" else
                                     f"compressed chunks 2^{w['c']}, eb={w['eb']}")
                + (f", psi checkpointed every {w['checkpoint']} forward pass(es)" if w.get("checkpoint") else ""))
    name = {"layers": f"random layered circuit depth {w.get('depth')}", "ghz": "GHZ", "qft": "QFT on a seeded basis state",
            "clifford": f"random Clifford+RZ depth {w.get('depth')} (40% of slots on the 10 high qubits)"}[w["circuit"]]
    bound = "relative eb" if w.get("relative") else "eb"
    return (f"{name}, n={w['n']} ({ngates} gates), {w['dtype']}, chunk=2^{w['c']}, {bound}={w['eb']}, compressed chunks "
            f"in pinned host DRAM, streamed in groups of "
            + (f"2^{group} chunks" if group is not None else
               (f"2^{w['group']} chunks" if w.get("group") else "chunks (group size chosen from the free HBM)")))


# ------------------------------------------------------------ distributed
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("BENCH_BACKEND", "nccl")
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max_sum(world, t_local: float, units_local: float, device=None):
    """(max over ranks of the step time, sum over ranks of the units)."""
    if world == 1:
        return t_local, units_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int = 0):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def host_link_peak():
    """Pinned bulk-copy bandwidth per direction and both at once (GB/s)."""
    import torch
    nbytes = 1 << 30
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d2 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = {}
    for name in ("h2d", "d2h"):
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s1):
                e0.record(s1)
                if name == "h2d":
                    d.copy_(h, non_blocking=True)
                else:
                    h.copy_(d, non_blocking=True)
                e1.record(s1)
            e1.synchronize()
            best = max(best, nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        out[name] = round(best, 1)
    best = 0.0
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, 2 * nbytes / (time.perf_counter() - t0) / 1e9)
    out["bidir"] = round(best, 1)
    del h, h2, d, d2
    torch.cuda.empty_cache()
    return out


def load_traffic(kind, alg_bytes_per_launch):
    """DRAM bytes per launch of the dominant kernel: the committed ncu capture's
    measured / algorithmic byte ratio (taken on a smaller launch of the same
    kernel; traffic grows with the amplitudes processed) applied to this run's
    algorithmic bytes per launch; None without a capture."""
    path = os.path.join(ROOT, "profiles", f"traffic_k_{kind}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    return int(alg_bytes_per_launch * t["bytes_per_amplitude"] / t["algorithmic_bytes_per_amplitude"])


def roofline_from_stats(d, n=None, amp_bytes=None, step_s=None, link=None, steps=1):
    """Roofline of the dominant kernel from one profiled step's counters.

    Top level (achieved, frac): the per-pass accounting, where a pass over
    the state owes 2 * 2^n * s bytes of HBM traffic however many tile sweeps
    it takes (fused gates ride free); one launch is credited its share,
    passes * 2 * 2^n * s / launches. "per_sweep" credits every tile sweep
    with the amplitudes it reads and writes (the kernel's own streaming
    rate). "step_binding": the slowest of the step's host-link and HBM terms
    against the measured step time."""
    hbm_peak, peak_kind = measured_peaks()
    kinds = {"apply": ("t_apply_s", "n_apply", "alg_bytes_apply"),
             "decode": ("t_decode_s", "n_decode", "alg_bytes_decode"),
             "encode": ("t_encode_s", "n_encode", "alg_bytes_encode")}
    total = sum(d[v[0]] for v in kinds.values())
    top = max(kinds, key=lambda k: d[kinds[k][0]])
    tk, nk, bk = kinds[top]
    launches = max(1, d[nk])
    avg_s = d[tk] / launches
    sweep_bytes = d[bk] / launches
    sweep_achieved = sweep_bytes / avg_s / 1e9 if avg_s > 0 else 0.0
    out = {"bound": "hbm", "unit": "GB/s", "peak": hbm_peak,
           "kernel": ("svj (generated sub-pass kernels)" if top == "apply" and d.get("jit_launches", 0) > 0
                      else f"k_{top}"),
           "peak_source": f"{peak_kind} (copy)", "launches": int(d[nk]), "avg_launch_ms": round(avg_s * 1e3, 4),
           "share_of_kernel_time": {k: round(d[v[0]] / max(1e-12, total), 3) for k, v in kinds.items()},
           "per_sweep": {"alg_bytes_per_launch": int(sweep_bytes), "achieved": round(sweep_achieved, 1),
                         "frac": round(sweep_achieved / hbm_peak, 4)}}
    if top == "apply" and n is not None and amp_bytes is not None and d["passes"] > 0:
        pass_bytes = d["passes"] * 2.0 * (1 << n) * amp_bytes
        per_launch = pass_bytes / launches
        ach = per_launch / avg_s / 1e9 if avg_s > 0 else 0.0
        out.update({"achieved": round(ach, 1), "frac": round(ach / hbm_peak, 4), "accounting": "per pass",
                    "alg_bytes_per_launch": int(per_launch), "sweeps_per_pass": round(launches / d["passes"], 2)})
        out["traffic"] = load_traffic(top, sweep_bytes)
    else:
        out.update({"achieved": round(sweep_achieved, 1), "frac": round(sweep_achieved / hbm_peak, 4),
                    "accounting": "per sweep", "alg_bytes_per_launch": int(sweep_bytes),
                    "traffic": load_traffic(top, sweep_bytes)})
    if step_s and n is not None:
        terms = {}
        if link:
            terms["h2d_ms"] = d["bytes_h2d"] / steps / (link["h2d"] * 1e9) * 1e3
            terms["d2h_ms"] = d["bytes_d2h"] / steps / (link["d2h"] * 1e9) * 1e3
        hbm = (d["passes"] / steps) * 2.0 * (1 << n) * amp_bytes if amp_bytes else 0.0
        if d["bytes_h2d"]:
            hbm += (d["bytes_h2d"] + d["bytes_d2h"]) / steps
        terms["hbm_ms"] = hbm / (hbm_peak * 1e9) * 1e3
        bind = max(terms, key=terms.get)
        out["step_binding"] = {"terms_ms": {k: round(v, 2) for k, v in terms.items()}, "binding": bind,
                               "measured_step_ms": round(step_s * 1e3, 2),
                               "frac": round(terms[bind] / (step_s * 1e3), 4)}
    return out


STAT_KEYS = ("passes", "subpasses", "groups", "kernel_launches", "bytes_h2d", "bytes_d2h", "t_decode_s", "t_apply_s",
             "t_encode_s", "n_decode", "n_apply", "n_encode", "alg_bytes_decode", "alg_bytes_apply",
             "alg_bytes_encode", "jit_launches", "t_h2d_s", "t_d2h_s", "t_encode_finish_s", "t_host_prepare_s",
             "t_host_wait_s", "remap_swaps")


# ------------------------------------------------------------ our arm
def run_apply(args, rank, world):
    import torch
    from paper_2309_16979_gb300 import StateVector

    w = args.w
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    n, c = w["n"], w["c"]
    gates = make_circuit(w, seed=1 + rank)
    terms = W.ising(n, seed=4)
    units_per_step = W.amp_gate_updates(n, gates)
    link = host_link_peak() if rank == 0 else None
    init = W.basis_index(n)

    # timed steps run without per-launch events; one extra profiled step after
    # them gives the kernel breakdown and the roofline
    def make_sim():
        return StateVector(n, c, w["eb"], dtype=w["dtype"], init_index=init, max_group_qubits=w["group"],
                           profile=False, relative_bound=bool(w.get("relative", False)),
                           host_budget_bytes=host_budget(), device=dev, jit=bool(args.jit),
                           remap_qubits=args.remap)

    if args.remap:
        # every remapped call leaves qubits on new positions, so the next call
        # runs other physical gates: a first handle makes the same sequence of
        # calls to compile all their kernels (process-wide cache) before the
        # timed handle starts
        with make_sim() as pre:
            for _ in range(args.warmup + args.steps + 1 + max(1, min(2, args.steps))):
                pre.apply(gates)
    sim = make_sim()
    group = sim.stats()["group_qubits"]  # resolved (0 = chosen from the free device memory)
    for _ in range(args.warmup):
        sim.apply(gates)
    s0 = sim.stats()
    clocks = ClockSampler(dev)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.apply(gates)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_local = e0.elapsed_time(e1) * 1e-3
    s1 = sim.stats()
    t_max, units = reduce_max_sum(world, t_local, units_per_step * args.steps, device="cuda")
    value = units / t_max
    d = {k: s1[k] - s0[k] for k in STAT_KEYS}
    link_bytes = d["bytes_h2d"] + d["bytes_d2h"]
    per_step = {k: d[k] / args.steps for k in ("passes", "subpasses", "kernel_launches", "bytes_h2d", "bytes_d2h",
                                                "remap_swaps")}
    # the profiled step (per-launch CUDA events on the library's streams)
    sim.set_profile(True)
    sp0 = sim.stats()
    sim.apply(gates)
    sp1 = sim.stats()
    sim.set_profile(False)
    dp = {k: sp1[k] - sp0[k] for k in STAT_KEYS}
    amp_bytes = 8 if w["dtype"] == "c64" else 16
    roofline = roofline_from_stats(dp, n=n, amp_bytes=amp_bytes, step_s=t_max / args.steps, link=link)

    # e2e: the public calls a user makes (apply + read back <H>), host buffers,
    # every H2D / D2H of the compressed store inside the timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_steps = max(1, min(2, args.steps))
    sa = sim.stats()
    energy = None
    for _ in range(e_steps):
        sim.apply(gates)
        energy = sim.expect(terms)
    te = (time.perf_counter() - t0) / e_steps
    sb = sim.stats()
    e2e = {"value": units_per_step * world / te, "unit": METRIC,
           "h2d_bytes_per_step": int((sb["bytes_h2d"] - sa["bytes_h2d"]) / e_steps),
           "d2h_bytes_per_step": int((sb["bytes_d2h"] - sa["bytes_d2h"]) / e_steps + 8),
           "includes": f"sv_apply_circuit + sv_expect(1-D Ising, {len(terms)} terms) with the energy read back"}
    st = sim.stats()
    gpu_launches = int(d["kernel_launches"])
    sim.close()
    default = args.workload == "layers30" and all(v is None for v in (args.eb, args.n, args.chunk, args.depth,
                                                                      args.group))
    # the same workload with one group holding every chunk (one pass per call)
    single = n - c if default and 2 <= n - c <= 8 and not args.remap else None
    quality = state_quality(w, gates, terms, dev, args.remap, extra_groups=(single,) if single else ()) \
        if rank == 0 and not args.no_extras else {}

    out = {
        "metric": METRIC, "value": value, "unit": "amp-gate updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{w['dtype']} (FP32 gate arithmetic for c64, FP64 reductions)"
        if w["dtype"] == "c64" else "c128 (FP64)", "data": "synthetic",
        "config": {"workload": describe(w, len(gates), group) + (", qubit remapping" if args.remap else ""),
                   "n_qubits": n, "chunk_qubits": c, "remap_qubits": bool(args.remap),
                   "abs_error_bound": w["eb"], "group_qubits": group, "gates": len(gates),
                   "l2": "inputs larger than L2: every pass streams the whole state; groups of 2^(c+g) amplitudes",
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": gpu_launches,
        "kernels": {"generated": bool(args.jit), "compiled": st["jit_kernels_compiled"],
                    "compile_s_before_timing": round(st["t_jit_compile_s"], 3),
                    "generated_launches_per_step": d["jit_launches"] / args.steps},
        "roofline": roofline,
        "e2e": e2e,
        "clocks": clk,
        "host_link": {"achieved_gbs": round(link_bytes / t_local / 1e9, 1), "peak_gbs": link,
                      "frac_of_bidir": round(link_bytes / t_local / 1e9 / link["bidir"], 3) if link else None,
                      "per_step": per_step},
        # per step, ms: kernel and copy durations (CUDA events on their streams; copies
        # overlap kernels) and host time planning / blocked on the GPU
        "breakdown_ms_per_step": {k: round(dp[v] * 1e3, 2) for k, v in (
            ("apply", "t_apply_s"), ("decode", "t_decode_s"), ("encode", "t_encode_s"),
            ("encode_finish", "t_encode_finish_s"), ("h2d", "t_h2d_s"), ("d2h", "t_d2h_s"),
            ("host_prepare", "t_host_prepare_s"), ("host_wait", "t_host_wait_s"))},
        "stored_state": {"compressed_bytes": st["compressed_bytes"], "raw_bytes": st["raw_bytes"],
                         "ratio": round(st["raw_bytes"] / max(1, st["compressed_bytes"]), 2),
                         "norm2": st["norm2"], "energy": energy,
                         "note": "after every warm-up, timed, profiled and e2e application of the circuit "
                                 "to the same handle: error compounds per pass"},
    }
    if quality:
        out["fidelity"] = quality["one_apply_vs_fp64"]
    if rank == 0 and not args.no_extras and w["n"] <= 32:
        out.update(comparator(args, gates, terms, energy, applies=args.warmup + args.steps + 1 + e_steps))
    if rank == 0 and not args.no_extras and single:
        out["single_group"] = single_group_leg(args, w, gates, units_per_step, single, dev,
                                               quality.get("one_apply_vs_fp64", {}).get(f"group_qubits_{single}"))
    if rank == 0 and not args.no_extras and default:
        out["adjoint_grad_s_per_step"] = adjoint_legs(dev)
    return out


def single_group_leg(args, w, gates, units_per_step, g, dev, quality):
    """The headline workload with max_group_qubits = n - c: one group holds
    every chunk, so each call is one pass (all chunks in, the fused sweeps,
    all chunks out) instead of several passes of 2^g-chunk groups streamed
    through a copy / compute pipeline. Timed like the headline (CUDA events
    over the same steps after the same warm-up)."""
    import torch
    from paper_2309_16979_gb300 import StateVector
    n, c = w["n"], w["c"]
    try:
        with StateVector(n, c, w["eb"], dtype=w["dtype"], init_index=W.basis_index(n), max_group_qubits=g,
                         host_budget_bytes=host_budget(), device=dev, jit=bool(args.jit)) as sim:
            for _ in range(args.warmup):
                sim.apply(gates)
            s0 = sim.stats()
            torch.cuda.synchronize()
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                sim.apply(gates)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3 / args.steps
            s1 = sim.stats()
        return {"value": units_per_step / t, "unit": METRIC, "ms_per_step": t * 1e3, "group_qubits": g,
                "passes_per_step": (s1["passes"] - s0["passes"]) / args.steps,
                "subpasses_per_step": (s1["subpasses"] - s0["subpasses"]) / args.steps,
                "one_apply_vs_fp64": quality}
    except Exception as ex:  # noqa: BLE001 -- reported, not hidden
        return {"error": str(ex)}


def state_quality(w, gates, terms, dev, remap=False, extra_groups=()):
    """Error of one application of the workload's circuit to its seeded basis
    state (a fresh handle, as a user's first call), against an FP64
    reference: the uncompressed complex128 GPU path (pinned to the FP64
    oracle at 1e-12 relative L2) where 2^n complex128 amplitudes fit in HBM,
    else the GHZ closed form. Reports the fidelity |<ref|psi>|^2 /
    (||ref||^2 ||psi||^2), the Ising energy error and the stored norm^2 of
    the compressed path, and the same for the plain uncompressed path in the
    workload's own precision (the comparator "at fidelity"); extra_groups:
    group sizes whose compressed path is measured the same way."""
    from paper_2309_16979_gb300 import StateVector
    n = w["n"]
    init = W.basis_index(n)
    kw = dict(dtype=w["dtype"], max_group_qubits=w["group"], device=dev,
              relative_bound=bool(w.get("relative", False)), host_budget_bytes=host_budget(), remap_qubits=remap)
    out = {"reference": None}
    if w["circuit"] == "ghz":
        with StateVector(n, w["c"], w["eb"], **kw) as s:
            s.apply(gates)
            a = s.amplitudes([0, (1 << n) - 1])
            st = s.stats()
        out.update({"reference": "GHZ closed form",
                    "fidelity": float(abs((a[0] + a[1]) / math.sqrt(2)) ** 2 / max(st["norm2"], 1e-300)),
                    "norm2": st["norm2"], "passes": st["passes"]})
        return {"one_apply_vs_fp64": out}
    if n > 30:
        return {"one_apply_vs_fp64": beyond_hbm_quality(w, gates, dev, kw)}
    t0 = time.perf_counter()
    with StateVector(n, mode="uncompressed", dtype="c128", init_index=init, device=dev) as ref:
        ref.apply(gates)
        e_ref = ref.expect(terms)
        with StateVector(n, w["c"], w["eb"], init_index=init, **kw) as s:
            s.apply(gates)
            st = s.stats()
            e_c = s.expect(terms)
            nr = ref.inner(ref).real
            dot, ns = s.inner(ref), st["norm2"]  # <psi|ref>; the stored state's exact FP64 norm^2
        comp = {"fidelity": float(abs(dot) ** 2 / max(nr * ns, 1e-300)), "infidelity": None,
                "energy": e_c, "energy_abs_err": abs(e_c - e_ref), "norm2": st["norm2"], "passes": st["passes"],
                "per_pass_infidelity_estimate": (2.0 / 3.0) * (1 << n) * w["eb"] ** 2
                if not w.get("relative") else None}
        comp["infidelity"] = 1.0 - comp["fidelity"]
        extra = {}
        for g in extra_groups:
            with StateVector(n, w["c"], w["eb"], init_index=init, **dict(kw, max_group_qubits=g)) as s:
                s.apply(gates)
                st = s.stats()
                e_g = s.expect(terms)
                dot, ns = s.inner(ref), st["norm2"]
            f = float(abs(dot) ** 2 / max(nr * ns, 1e-300))
            extra[f"group_qubits_{g}"] = {"fidelity": f, "infidelity": 1.0 - f, "energy": e_g,
                                          "energy_abs_err": abs(e_g - e_ref), "passes": st["passes"]}
        with StateVector(n, mode="uncompressed", dtype=w["dtype"], init_index=init, device=dev) as p:
            p.apply(gates)
            e_p = p.expect(terms)
            dot, npl = p.inner(ref), p.inner(p).real
        plain = {"fidelity": float(abs(dot) ** 2 / max(nr * npl, 1e-300)), "energy": e_p,
                 "energy_abs_err": abs(e_p - e_ref), "norm2": npl}
        plain["infidelity"] = 1.0 - plain["fidelity"]
    out.update({"reference": "uncompressed complex128 GPU path", "reference_energy": e_ref,
                "compressed": comp, "plain_uncompressed": plain, **extra,
                "seconds": round(time.perf_counter() - t0, 1)})
    return {"one_apply_vs_fp64": out}


def beyond_hbm_quality(w, gates, dev, kw, samples=4096):
    """Fidelity where no FP64 reference state fits anywhere (2^n complex128
    amplitudes above HBM and host memory): the circuit and then its inverse
    from the seeded basis state |x>, F = |<x|psi>|^2 / ||psi||^2 (every pass
    of both halves re-quantises the state); for QFT also the amplitudes of
    one application at seeded sample indices against the closed form
    2^(-n/2) exp(2 pi i x k / 2^n), with the overlap they estimate."""
    from paper_2309_16979_gb300 import StateVector
    n = w["n"]
    x = W.basis_index(n)
    out = {"reference": "circuit then inverse back to the basis state"
           + ("; QFT closed form at sampled amplitudes" if w["circuit"] == "qft" else "")}
    t0 = time.perf_counter()
    with StateVector(n, w["c"], w["eb"], init_index=x, **kw) as s:
        s.apply(gates)
        st = s.stats()
        out["one_apply"] = {"passes": st["passes"], "norm2": st["norm2"], "compressed_bytes": st["compressed_bytes"],
                            "host_pinned_bytes": st["host_pinned_bytes"],
                            "ratio": round(st["raw_bytes"] / max(1, st["compressed_bytes"]), 2)}
        if w["circuit"] == "qft":
            rng = W.SplitMix64(7)
            idx = [rng.next_u64() % (1 << n) for _ in range(samples)]
            a = s.amplitudes(idx)
            ref = np.array([np.exp(2j * np.pi * ((x * k) % (1 << n)) / (1 << n)) for k in idx]) * 2.0 ** (-n / 2)
            err = np.abs(a - ref) / 2.0 ** (-n / 2)
            est = abs(np.vdot(ref, a)) ** 2 / (np.vdot(ref, ref).real * np.vdot(a, a).real)
            out["one_apply"].update({"sampled_amplitudes": samples, "max_rel_err": float(err.max()),
                                     "rms_rel_err": float(np.sqrt(np.mean(err ** 2))),
                                     "fidelity_estimate_from_samples": float(est)})
        s.apply(W.inverse(gates))
        st2 = s.stats()
        ax = s.amplitudes([x])[0]
        out["circuit_then_inverse"] = {"passes": st2["passes"], "norm2": st2["norm2"],
                                       "fidelity": float(abs(ax) ** 2 / max(st2["norm2"], 1e-300))}
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def comparator(args, gates, terms, energy_c, applies):
    """The plain uncompressed in-HBM GPU path on the same circuit, and the
    FP64 oracle on a bounded sample of the workload."""
    import torch
    from paper_2309_16979_gb300 import StateVector
    w = args.w
    out = {}
    n = w["n"]
    units = W.amp_gate_updates(n, gates)
    try:
        with StateVector(n, mode="uncompressed", dtype=w["dtype"], init_index=W.basis_index(n), profile=False,
                         jit=bool(args.jit)) as p:
            for _ in range(applies):
                p.apply(gates)
            e_plain = p.expect(terms)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.apply(gates)
            t = time.perf_counter() - t0
            p.set_profile(True)  # the roofline from one more, profiled, apply
            s0 = p.stats()
            p.apply(gates)
            s1 = p.stats()
        d = {k: s1[k] - s0[k] for k in STAT_KEYS}
        out["plain_uncompressed"] = {"value": units / t, "unit": METRIC, "seconds_per_step": t,
                                     "subpasses_per_step": d["subpasses"],
                                     "roofline": roofline_from_stats(d, n=n, amp_bytes=8 if w["dtype"] == "c64" else 16,
                                                                     step_s=t),
                                     "energy_after_same_applies": e_plain, "energy_compressed": energy_c,
                                     "energy_abs_diff": abs(e_plain - energy_c) if energy_c is not None else None}
    except Exception as ex:  # noqa: BLE001
        out["plain_uncompressed"] = {"error": str(ex)}
    out["cpu_baseline"] = cpu_baseline(w, gates)
    return out


def oracle_sample(n, gates, psi, first, target_s, threads=None):
    """The one sampling protocol of both bench arms: the FP64 oracle (as it
    stands) applies consecutive gates of the workload, starting at gate
    `first`, to the full 2^n complex128 state, as many as fit in about
    target_s (timed by the first of them); returns (state, gates applied,
    seconds, threads used)."""
    import oracle
    if threads:
        oracle.set_num_threads(threads)
    used = oracle.num_threads()
    t0 = time.perf_counter()
    psi = oracle.apply_gates(n, psi, [gates[first % len(gates)]], inplace=True)
    t1 = time.perf_counter() - t0
    k = max(1, int(target_s / max(t1, 1e-4)) - 1)
    sample = [gates[(first + 1 + j) % len(gates)] for j in range(k)]
    t0 = time.perf_counter()
    psi = oracle.apply_gates(n, psi, sample, inplace=True)
    dt = time.perf_counter() - t0 + t1
    return psi, k + 1, dt, used


def cpu_baseline(w, gates, target_s=10.0):
    """FP64 oracle on the host cores, all of them and one: consecutive gates
    of the workload on the full n-qubit complex128 state; amp-gate updates/s."""
    import oracle
    n = w["n"]
    psi = oracle.basis_state(n, W.basis_index(n))
    all_cores = oracle.num_threads()
    psi, k, dt, used = oracle_sample(n, gates, psi, 0, target_s)
    _, k1, dt1, _ = oracle_sample(n, gates, psi, k, target_s / 2, threads=1)
    oracle.set_num_threads(all_cores)
    return {"value": k * (1 << n) / dt, "unit": METRIC, "cores": used, "kind": "oracle",
            "sample": f"gates 1..{k} of the {len(gates)}-gate workload on the full 2^{n} complex128 state "
                      f"({dt:.1f} s on {used} threads)",
            "single_thread": {"value": k1 * (1 << n) / dt1, "cores": 1,
                              "sample": f"gates {k + 1}..{k + k1} ({dt1:.1f} s)"}}


def grad_measure(w, steps, warmup, dev, world=1, with_errors=True, max_sets=None):
    """Adjoint gradient seconds per step on an HEA workload, and every timed
    set's energy and gradient error against the FP64 reference (the
    uncompressed complex128 GPU adjoint, pinned to the FP64 oracle)."""
    import torch
    from paper_2309_16979_gb300 import StateVector
    n = w["n"]
    gates, npar = W.hea(n, w["layers"])
    terms = W.ising(n, seed=4)
    sets = w.get("sets", 1) if max_sets is None else min(max_sets, w.get("sets", 1))
    thetas = [W.normal_params(npar, seed=(3 if w.get("sets", 1) == 1 else 100 + i)) for i in range(max(1, sets))]
    mode = w.get("mode", "compressed")
    sim = StateVector(n, w["c"], w["eb"] or 1e-6, dtype=w["dtype"], mode=mode, max_group_qubits=w["group"], device=dev,
                      host_budget_bytes=host_budget() if mode == "compressed" else 0,
                      checkpoint_passes=w.get("checkpoint", 0))
    for i in range(warmup):
        sim.grad(gates, thetas[i % len(thetas)], terms)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(dev)
    clocks.start()
    s0 = sim.stats()
    t0 = time.perf_counter()
    results = []
    for i in range(steps):
        results.append(sim.grad(gates, thetas[i % len(thetas)], terms))
    torch.cuda.synchronize()
    t_local = (time.perf_counter() - t0) / steps
    clk = clocks.stop()
    barrier(world)
    st = sim.stats()
    launches = int(st["kernel_launches"] - s0["kernel_launches"])
    adj_launches = int(st["jit_adjoint_launches"] - s0["jit_adjoint_launches"])
    passes = (st["passes"] - s0["passes"]) / steps
    ckpt = {"checkpoint_passes": w.get("checkpoint", 0), "checkpoints": st["checkpoints"],
            "checkpoint_bytes": st["checkpoint_bytes"]}
    sim.close()
    errors = []
    if with_errors:
        ref = StateVector(n, mode="uncompressed", dtype="c128", device=dev)
        for i in range(min(steps, len(thetas))):
            e_r, g_r = ref.grad(gates, thetas[i], terms)
            e, g = results[i]
            errors.append({"set": i, "energy": e, "energy_err": abs(e - e_r),
                           "grad_max_err": float(np.abs(g - g_r).max()),
                           "grad_rel_l2": float(np.linalg.norm(g - g_r) / max(np.linalg.norm(g_r), 1e-300))})
        ref.close()
    return {"s_per_step": t_local, "steps": steps, "warmup": warmup, "params": npar, "gates": len(gates),
            "group_qubits": st["group_qubits"],
            "last_step_s": {k: round(st[f"t_grad_{k}_s"], 4) for k in ("forward", "lambda", "reverse")}
            if mode == "compressed" else None,
            "parameter_sets": len(thetas), "launches_per_step": launches / steps,
            "generated_adjoint_launches_per_step": adj_launches / steps, "passes_per_step": passes,
            "clocks": clk, "errors_vs_fp64_gpu_adjoint": errors, "workload": describe(w, len(gates)), **ckpt}


def run_grad(args, rank, world):
    """Adjoint gradient seconds per step (the HEA workloads: n = 24 in HBM, n = 32 compressed)."""
    import torch
    w = args.w
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    m = grad_measure(w, args.steps, args.warmup, dev, world, with_errors=not args.no_extras and rank == 0)
    t_max, _ = reduce_max_sum(world, m["s_per_step"], 1.0, device="cuda")
    return {"metric": "adjoint grad s/step", "value": t_max, "unit": "s/step", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic",
            "config": {"workload": m["workload"], "n_qubits": w["n"], "params": m["params"], "gates": m["gates"],
                       "parameter_sets": m["parameter_sets"], "parallelism": f"replicas x{world}"},
            "gpu_launches": int(m["launches_per_step"] * args.steps), "clocks": m["clocks"],
            "passes_per_step": m["passes_per_step"], "group_qubits": m["group_qubits"],
            "last_step_s": m["last_step_s"],
            "generated_adjoint_launches_per_step": m["generated_adjoint_launches_per_step"],
            "errors_vs_fp64_gpu_adjoint": m["errors_vs_fp64_gpu_adjoint"]}


def adjoint_legs(dev):
    """The metric's second part, adjoint gradient seconds per step, on the two
    gradient workloads: n = 24 in HBM (480 parameters) and n = 32 on two
    compressed stores (512 parameters; two of its 16 parameter sets)."""
    out = {}
    # warm-up covers every parameter set the timed steps use: a gate's kernel
    # depends on which matrix entry it is scaled by, which can change with
    # the angles, so a new set may compile kernel variants once
    for name, steps, warmup, max_sets in (("grad-hea24", 5, 2, None), ("grad-hea32", 2, 2, 2),
                                          ("grad-hea32-ckpt1", 2, 2, 2)):
        try:
            m = grad_measure(WORKLOADS[name], steps, warmup, dev, max_sets=max_sets)
            m.pop("clocks", None)
            out[name] = m
        except Exception as ex:  # noqa: BLE001 -- reported, not hidden
            out[name] = {"error": str(ex)}
    return out


# ------------------------------------------------------------- Table 1
# the paper's numbers (seconds; hardware and precision not stated)
PAPER_TABLE1 = {20: {"h2d": {"sync": 0.003, "async": 2.7, "buffer": 0.003},
                     "d2h": {"sync": 0.008, "async": 9.2, "buffer": 0.004}},
                25: {"h2d": {"sync": 0.080, "async": 77.9, "buffer": 0.110},
                     "d2h": {"sync": 0.233, "async": 294.4, "buffer": 0.273}}}


def run_table1(args):
    """Sync / async-per-amplitude / buffer+remap copies of a complex128 state
    (sv_copy_probe), median of 3 (async: the first 2^20 amplitudes timed,
    scaled to 2^n)."""
    from paper_2309_16979_gb300 import copy_probe
    rows, verified = [], True
    for n in (20, 25):
        row = {"n_qubits": n}
        for direction in ("h2d", "d2h"):
            row[direction] = {}
            for strategy in ("sync", "async", "buffer"):
                times = []
                for _ in range(1 if strategy == "async" else 3):
                    t, ok = copy_probe(n, strategy, direction, "c128", sample=1 << 20 if strategy == "async" else 0)
                    times.append(t)
                    verified = verified and ok
                row[direction][strategy] = sorted(times)[len(times) // 2]
            row[direction]["async_over_sync"] = row[direction]["async"] / row[direction]["sync"]
            row[direction]["buffer_over_sync"] = row[direction]["buffer"] / row[direction]["sync"]
        rows.append(row)
    return {"metric": "host<->device copy seconds (Table 1)", "unit": "s", "dtype": "c128", "data": "synthetic",
            "rows": rows, "all_amplitudes_verified": verified, "paper": PAPER_TABLE1,
            "note": "async copies the first 2^20 amplitudes one cudaMemcpyAsync each and scales to 2^n; "
                    "buffer = one bulk copy + a kernel moving every amplitude to its position"}


# ------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The FP64 CPU oracle as the reference arm, on the same config and metric,
    sampled as the cpu_baseline leg samples it (consecutive gates of the
    workload on the full state), about 2 s of gates per step."""
    import oracle
    w = args.w
    n = w["n"]
    gates = make_circuit(w, seed=1) if w["circuit"] != "hea" else W.hea(n, w["layers"])[0]
    psi = oracle.basis_state(n, W.basis_index(n))
    first, done, t, used = 0, 0, 0.0, oracle.num_threads()
    for i in range(args.warmup + args.steps):
        psi, k, dt, used = oracle_sample(n, gates, psi, first, 2.0)
        first += k
        if i >= args.warmup:
            done += k
            t += dt
    value = done * (1 << n) / t
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "amp-gate updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64)",
            "data": "synthetic",
            "config": {"workload": describe(w, len(gates)) + "; FP64 oracle on the host cores", "n_qubits": n},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": used, "kind": "oracle",
                             "sample": f"{done} consecutive gates of the {len(gates)}-gate workload over the timed "
                                       f"steps (about 2 s each) on the full 2^{n} complex128 state"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world = dist_init()
    if args.table1:
        if rank == 0:
            print(json.dumps(run_table1(args)), flush=True)
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    try:
        out = run_grad(args, rank, world) if args.w["circuit"] == "hea" else run_apply(args, rank, world)
    except Exception as exc:  # noqa: BLE001 -- reported, not hidden
        from paper_2309_16979_gb300._abi import SvError
        if not (isinstance(exc, SvError) and exc.code in (-6, -2)):
            raise
        w = args.w
        out = {"metric": METRIC, "value": None, "unit": "amp-gate updates/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic",
               "config": {"workload": describe(w, len(make_circuit(w, seed=1))), "n_qubits": w["n"],
                          "chunk_qubits": w["c"], "abs_error_bound": w["eb"]}}
        if exc.code == -6:
            # an absolute error bound above the amplitudes' magnitude quantises the
            # whole state to zero: a property of the bound, reported as such
            out["norm_collapse"] = {"error": str(exc),
                                    "reason": f"spread amplitudes (|a| ~ 2^-{w['n'] // 2}) fall below half the "
                                              f"quantisation step of eb={w['eb']} and quantise to zero"}
        else:
            # the compressed state outgrew the host memory the bench allows
            out["host_oom"] = {"error": str(exc), "host_budget_bytes": host_budget(),
                               "reason": "the stored state (two arenas) needs more pinned host memory"}
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
