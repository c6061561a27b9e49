#!/usr/bin/env python
"""Benchmark: KADABRA adaptive-sampling betweenness on one GB300.

Default workload: R-MAT scale 26 (2^26 vertices, edge factor 16, Graph500
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05)), symmetrised, self-loops and
duplicates removed, int64 offsets / int32 columns; eps = 0.01, delta = 0.1,
seed 1: the largest single-GPU configuration.  Synthetic data from
paper_1910_11039_gb300.inputs (generator seed 4).  --workload picks the other
single-query graphs (R-MAT scale 20, the 4096^2 grid, ...).

A step is one complete adaptive phase (arXiv 1910.11039, Section III-A,
phase 3): from tau = 0, epochs of E samples each checked against the stopping
condition, until it holds.  Default form ("pipelined"): one persistent launch
in which epochs flow through rotating frames and the CTA that completes an
epoch checks it while the others keep sampling (the paper's epoch framework,
Section IV).  Form "epochs": one sampling launch plus one stop-check launch
per epoch, all enqueued without host synchronisation (launches after the stop
take no samples).  The graph and the calibrated budgets are resident in HBM
before the timed region.  L2 is flushed (256 MiB write) before every step.

value  = adaptive samples per second over the K timed steps (device events)
e2e    = the same metric for whole queries through the C ABI from pinned host
         buffers: graph upload, diameter bound, calibration, adaptive phase,
         result download.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shortest-path samples/sec and time-to-(eps,delta) stop; GTEPS and HBM fraction"
WORKLOADS = {
    "rmat20": dict(graph="rmat20", eps=0.01, delta=0.1, seed=1, threads=512,
                   desc="R-MAT scale 20, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), symmetrised, "
                        "no self-loops/duplicates, int32 CSR; eps=0.01 delta=0.1 seed=1"),
    "rmat26": dict(graph="rmat26", eps=0.01, delta=0.1, seed=1, threads=1024, steps=20, e2e_steps=1,
                   cpu_samples=3200, ref_samples=1600, off64=True,
                   desc="R-MAT scale 26, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), symmetrised, "
                        "no self-loops/duplicates, int64 offsets / int32 columns; eps=0.01 delta=0.1 seed=1"),
    "rhg20": dict(graph="rhg20", eps=0.01, delta=0.1, seed=1, steps=5, cpu_samples=4800, ref_samples=1600, threads=512,
                  desc="random hyperbolic graph, n=2^20, power-law exponent 3, average degree 60 (|E| = 30|V|), "
                       "seed 20, int32 CSR; eps=0.01 delta=0.1 seed=1"),
    "grid4096": dict(graph="grid4096", eps=0.01, delta=0.1, seed=1, steps=1, e2e_steps=1, cpu_samples=48,
                     ref_samples=16,
                     desc="4096x4096 grid, 10% of the edges deleted (seed 3), largest component, int32 CSR; "
                          "eps=0.01 delta=0.1 seed=1"),
    "grid512": dict(graph="grid512", eps=0.05, delta=0.1, seed=1, steps=5, cpu_samples=1600, ref_samples=800,
                    desc="512x512 grid, 10% of the edges deleted (seed 3), largest component, int32 CSR; "
                         "eps=0.05 delta=0.1 seed=1 (small high-diameter case for profiles)"),
    "er2000": dict(graph="er2000", eps=0.05, delta=0.1, seed=1,
                   desc="Erdos-Renyi G(n=2000, avg degree 8) seed 1, largest component, int32 CSR; "
                        "eps=0.05 delta=0.1 seed=1"),
}
FLUSH_BYTES = 256 << 20
REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
               0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(g, seed, per_thread, threads, pool=None):
    """Run the oracle's sampler on `threads` host threads, each taking
    `per_thread` consecutive adaptive-phase sample indices on its own
    workspace (built before the timed region); returns
    (samples/s, samples, e_scan, seconds)."""
    import oracle
    oracle.build()
    pool = pool or [oracle.Workspace(g) for _ in range(threads)]
    results = [None] * threads

    def work(i):
        results[i] = pool[i].run_samples(seed, 1, i * per_thread, (i + 1) * per_thread)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(threads)]
    t0 = time.perf_counter()
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    dt = time.perf_counter() - t0
    samples = sum(r[1].samples for r in results)
    e_scan = sum(r[1].e_scan for r in results)
    return samples / dt, samples, e_scan, dt


def cpu_baseline_for(g, wl, args):
    """The oracle as it stands on the host cores: all-core and single-thread
    samples/s over bounded index ranges of the workload, and its time to the
    (eps, delta) stop with the benchmarked epoch length (the whole method,
    threads over each epoch's index range, then the oracle's check), measured
    when a bounded estimate says it ends within ~2 minutes, else extrapolated
    from the all-core rate and the stop tau."""
    import oracle
    cores = host_cores()
    pool = [oracle.Workspace(g) for _ in range(cores)]
    per = max(1, args.cpu_samples // cores)
    rate, s, e, dt = oracle_rate(g, wl["seed"], per, cores, pool)
    per1 = max(1, min(per, int(rate / cores * 4) or 1))
    rate1, s1, _, dt1 = oracle_rate(g, wl["seed"], per1, 1, pool[:1])
    del pool
    out = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
           "sample": f"adaptive-phase sample indices [0, {s}) of the same workload, {per} per thread on {cores} "
                     f"threads ({dt:.1f} s wall); single thread: [0, {s1}) ({dt1:.1f} s)",
           "gteps": e / dt / 1e9, "single_thread": {"value": rate1, "unit": "samples/s", "threads": 1}}
    # the oracle's whole run: estimate the adaptive phase from omega's order first
    est = oracle.omega(wl["eps"], wl["delta"], oracle.vertex_diameter_bound(g)) / 2 / rate
    if est <= 120 and not args.no_oracle_stop:
        _, _, _, _, inf = oracle.kadabra_threads(g, wl["eps"], wl["delta"], seed=wl["seed"], epoch_len=args.epoch,
                                                 threads=cores)
        out["time_to_stop"] = {"value": inf["seconds"]["adaptive"], "unit": "s", "measured": True,
                               "tau": inf["tau"], "stop_epoch": inf["stop_epoch"],
                               "phases_1_2_s": inf["seconds"]["phases_1_2"], "threads": cores}
    else:
        out["time_to_stop"] = {"value": None, "unit": "s", "measured": False,
                               "estimate_from_rate": "stop tau / all-core samples/s (see the GPU line's samples_per_step)"}
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), int(parts[4], 16), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        busy = [r for r in rows if not (r[3] & 0x1)] or rows
        reasons = set()
        for r in busy:
            for bit, name in REASON_BITS.items():
                if r[3] & bit and bit != 0x1:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------

def algorithmic_bytes(ls, offset_bytes):
    """Bytes one launch must move at minimum: per expanded vertex its two row
    offsets, per scanned adjacency entry its 4-byte column id, per reached
    vertex a 16-byte state record (level + path count), per back-walk scan a
    column id, per counted interior vertex a 4-byte counter update."""
    return (2 * offset_bytes * ls.expanded + 4 * ls.e_scan + 16 * ls.touched + 4 * ls.walk_scan
            + 4 * ls.interior)


KERNEL_SOURCES = ("sample_kernel.cu", "philox.cuh", "stop_math.cuh")


def _code_only(text: str) -> str:
    """Source text without comments and blank lines (comment edits do not
    change the compiled kernel, so they must not invalidate a profile)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = []
    for line in text.splitlines():
        line = re.sub(r"//.*$", "", line).rstrip()
        if line.strip():
            lines.append(line)
    return "\n".join(lines)


def kernel_digest():
    """Digest of the code (comments stripped) the sampling kernels are compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_11039_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode() + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload, kernel):
    """DRAM bytes per sample of the timed kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"kernel_digest:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_sample:\s*([0-9.eE+]+)", txt)
    if not m or not b or m.group(1) != kernel_digest():
        return None
    return float(b.group(1))


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args, wl, g, rank, world):
    if rank != 0:
        return
    import oracle
    threads = host_cores()
    per_thread = max(1, args.ref_samples // threads)
    seed = wl["seed"]
    pool = [oracle.Workspace(g) for _ in range(threads)]
    for _ in range(args.warmup):
        oracle_rate(g, seed, max(1, per_thread // 4), threads, pool)
    rates, total_s, total_dt = [], 0, 0.0
    for k in range(args.steps):
        rate, s, e, dt = oracle_rate(g, seed, per_thread, threads, pool)
        rates.append(rate)
        total_s += s
        total_dt += dt
    value = total_s / total_dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["desc"], "name": args.workload, "n": g.n, "nnz": g.nnz},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per_thread} adaptive-phase samples per thread x {threads} threads per step"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, wl, g, rank, world, local_rank, cpu_baseline):
    import numpy as np
    import torch

    from paper_1910_11039_gb300 import build as B
    from paper_1910_11039_gb300 import kadabra as K

    B.build()
    K.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    seed = wl["seed"] + rank          # replicas: independent queries per rank
    eps, delta = wl["eps"], wl["delta"]

    # ---- device-resident arm ----
    off64 = bool(wl.get("off64")) or g.nnz >= 2**31
    G = K.Graph.from_inputs(g, offsets_64=off64, skip_validate=True)
    q = K.Query(G, eps=eps, delta=delta, seed=seed, slots=args.slots, threads=args.threads)
    info0 = q.info()
    E = args.epoch
    max_epochs = math.ceil(info0.omega_ceil / E) + 1
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def adaptive_phase(qq):
        if args.mode == "pipelined":
            qq.run_pipelined(E, frames=args.frames)
        else:
            for _ in range(max_epochs):
                qq.sample_epoch(E)
                qq.check_stop_async()

    def step():
        flush.fill_(rank + 1)
        q.reset()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        adaptive_phase(q)
        s1.record(stream)
        s1.synchronize()
        inf = q.info()
        return s0.elapsed_time(s1), inf

    for _ in range(args.warmup):
        step()
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = q.info().launches
    clocks = ClockSampler(local_rank)
    clocks.start()
    t_wall0 = time.perf_counter()
    times, taus, escans, stops = [], [], [], []
    for _ in range(args.steps):
        ms, inf = step()
        times.append(ms)
        taus.append(inf.tau)
        escans.append(inf.e_scan)
        stops.append(inf.stop_epoch)
        assert inf.stopped, "adaptive phase did not stop within the omega cap"
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    total_ms = sum(times)
    if dist:
        t = torch.tensor([total_ms, wall], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        s = torch.tensor([float(sum(taus)), float(sum(escans))], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(s, op=torch.distributed.ReduceOp.SUM)
        total_ms_max, wall_max = t.tolist()
        all_samples, all_escan = s.tolist()
        torch.distributed.barrier()
    else:
        total_ms_max, wall_max = total_ms, wall
        all_samples, all_escan = float(sum(taus)), float(sum(escans))
    value = all_samples / (total_ms_max / 1e3)
    gteps = all_escan / (total_ms_max / 1e3) / 1e9

    # roofline of the sampling kernel over the timed steps' launches
    timed = min(256, q.info().launches - launches0)
    launches = [ls for ls in q.launch_log(timed) if ls.samples > 0]
    ob = 8 if off64 else 4
    peak, peak_kind = measured_peak_hbm()
    tot_b = sum(algorithmic_bytes(ls, ob) for ls in launches)
    tot_ms = sum(ls.ms for ls in launches)
    achieved = tot_b / (tot_ms / 1e3) / 1e9 if tot_ms > 0 else 0.0
    per_sample = profiled_traffic(args.workload, "batch_kernel" if args.mode == "pipelined" else "sample_kernel")
    mean_samples = sum(ls.samples for ls in launches) / max(1, len(launches))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": per_sample * mean_samples if per_sample else None,
                "kernel": "batch_kernel" if args.mode == "pipelined" else "sample_kernel", "peak_source": f"{peak_kind} hbm_gbs",
                "launches": len(launches), "avg_launch_ms": tot_ms / max(1, len(launches)),
                "algorithmic_bytes_per_launch": tot_b / max(1, len(launches)),
                "per_sample": {k: sum(getattr(ls, k) for ls in launches) / max(1, sum(ls.samples for ls in launches))
                               for k in ("e_scan", "expanded", "touched", "walk_scan", "interior", "connected")}}
    # our kernels per step: the query reset, then (pipelined: pipeline begin, class
    # maxima and one persistent launch; epochs: one sampling and one check launch
    # per enqueued epoch)
    n_launch_kernels = args.steps * (4 if args.mode == "pipelined" else 2 * max_epochs + 1)

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        off_np = g.offsets if off64 else g.offsets32()
        off_h = torch.from_numpy(off_np).pin_memory()
        col_h = torch.from_numpy(g.cols).pin_memory()
        b_h = torch.empty(g.n, dtype=torch.float64).pin_memory()
        c_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
        del q, G
        torch.cuda.synchronize()
        e_times, e_taus, e_phases = [], [], []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G2 = K.Graph(g.n, off_h.numpy(), col_h.numpy(), offsets_64=off64, skip_validate=True, stream=stream)
            stream.synchronize()
            ta = time.perf_counter()
            q2 = K.Query(G2, eps=eps, delta=delta, seed=seed, stream=stream, slots=args.slots, threads=args.threads)
            stream.synchronize()
            tb = time.perf_counter()
            if args.mode == "pipelined":
                q2.run_pipelined(E, frames=args.frames)
            else:
                for _ in range(math.ceil(q2.info().omega_ceil / E) + 1):
                    q2.sample_epoch(E)
                    q2.check_stop_async()
            stream.synchronize()
            tc = time.perf_counter()
            tau, se = q2.result_into(b_h.data_ptr(), c_h.data_ptr())
            t1 = time.perf_counter()
            q2.free()
            G2.free()
            if k > 0:      # the first query warms allocator and caches
                e_times.append(t1 - t0)
                e_taus.append(tau)
                e_phases.append((ta - t0, tb - ta, tc - tb, t1 - tc))
        n = g.n
        h2d = off_np.nbytes + g.cols.nbytes + 16 * n
        d2h = 4 * n + 8 * n + 4 * n
        e2e = {"value": sum(e_taus) / sum(e_times), "unit": "samples/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": len(e_times),
               "time_to_stop_ms": 1e3 * statistics.mean(e_times),
               "step": "graph upload + diameter bound + calibration + adaptive phase + result download",
               "phases_ms": {name: 1e3 * statistics.mean(p[i] for p in e_phases) for i, name in
                             enumerate(("graph_load", "query_create_calibrate", "adaptive", "result_download"))}}

    if rank != 0:
        return
    if cpu_baseline and not cpu_baseline["time_to_stop"].get("measured"):
        cpu_baseline["time_to_stop"]["value"] = (all_samples / args.steps / world) / cpu_baseline["value"]
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["desc"], "name": args.workload, "n": g.n, "nnz": g.nnz, "epoch_len": E,
                   "mode": args.mode, "frames": args.frames if args.mode == "pipelined" else None,
                   "max_epochs_enqueued": max_epochs if args.mode == "epochs" else None,
                   "slots": info0.slots, "threads": info0.threads,
                   "omega": info0.omega, "vertex_diameter": info0.vertex_diameter, "n_calib": info0.n_calib,
                   "l2": "flushed before every step (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "time_to_stop_ms": total_ms_max / args.steps,
        "samples_per_step": all_samples / args.steps / world,
        "stop_epoch": stops[-1],
        "gteps": gteps,
        "roofline": roofline,
        "cpu_baseline": cpu_baseline,
        "e2e": e2e,
        "gpu_launches": n_launch_kernels,
        "clocks": clk,
        "wall_s": wall_max,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# one query sharded over the ranks: epoch logs exchanged, two frames
# ---------------------------------------------------------------------------

def run_sharded(args, wl, g, rank, world, local_rank):
    """Every rank takes its share of each epoch's sample indices (a contiguous
    range), samples it into an epoch log on a side stream while the previous
    epoch's logs are all-gathered, folded and checked on every rank (the
    paper's epoch aggregation, Section IV, with logs instead of counter
    vectors).  value = the query's samples (tau at the stop) per second of the
    slowest rank; the work per step is fixed, so the scaling is strong."""
    import torch
    import torch.distributed as dist

    from paper_1910_11039_gb300 import build as B
    from paper_1910_11039_gb300 import kadabra as K
    from paper_1910_11039_gb300.distributed import LibraryShard, ShardedRun

    B.build()
    K.load()
    dev = torch.device("cuda", local_rank)
    off64 = bool(wl.get("off64")) or g.nnz >= 2**31
    G = K.Graph.from_inputs(g, offsets_64=off64, skip_validate=True)
    q = K.Query(G, eps=wl["eps"], delta=wl["delta"], seed=wl["seed"], slots=args.slots, threads=args.threads)
    info0 = q.info()
    E = args.epoch
    share = -(-E // world)
    shard = LibraryShard(q, device=dev, log_cap=share * max(1, info0.vertex_diameter))
    runner = ShardedRun(shard, shard, info0.omega_ceil, dist)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        flush.fill_(1)
        q.reset()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stopped, tau, epochs = runner.run_logs(E)
        e1.record(stream)
        e1.synchronize()
        assert stopped
        return e0.elapsed_time(e1), tau, epochs

    for _ in range(args.warmup):
        step()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    times, taus = [], []
    for _ in range(args.steps):
        ms, tau, epochs = step()
        times.append(ms)
        taus.append(tau)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t = torch.tensor([sum(times)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    dist.barrier()
    if rank != 0:
        return
    samples = float(sum(taus))
    line = {
        "metric": METRIC, "value": samples / (total_ms / 1e3), "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["desc"], "name": args.workload, "n": g.n, "nnz": g.nnz, "epoch_len": E,
                   "mode": "sharded", "threads": info0.threads, "slots": info0.slots,
                   "l2": "flushed before every step (256 MiB write)",
                   "parallelism": f"one query sharded over {world} rank(s): epoch logs all-gathered, two frames"},
        "time_to_stop_ms": total_ms / args.steps, "samples_per_step": samples / args.steps,
        "stop_epoch": epochs - 1, "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# many queries of uneven size: one persistent launch vs one launch per query
# ---------------------------------------------------------------------------

BATCHED_DESC = ("64 graphs: 56 R-MAT (scale U{12..18}, edge factor U{8..32}, Graph500 (a,b,c,d), symmetrised, "
                "no self-loops/duplicates) + 8 random geometric graphs (n U[50k,500k], unit square, radius "
                "sqrt(10/(pi n))), graph i generated from seed 1000+i, int32 CSR; per query eps=0.02 delta=0.1 "
                "seed=1000+i")


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * p / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def tts_summary(ms, samples, tts):
    return {"makespan_ms": ms, "samples_per_s": samples / (ms / 1e3), "tts_p50_ms": percentile(tts, 50),
            "tts_p99_ms": percentile(tts, 99), "tts_max_ms": max(tts)}


def run_batched(args, local_rank):
    import numpy as np
    import torch

    from paper_1910_11039_gb300 import autotune as AT
    from paper_1910_11039_gb300 import build as B
    from paper_1910_11039_gb300 import inputs
    from paper_1910_11039_gb300 import kadabra as K

    t0 = time.perf_counter()
    specs = inputs.batched_specs()
    graphs = [inputs.graph_from_spec(sp, f"mix{i}") for i, sp in enumerate(specs)]
    gen_s = time.perf_counter() - t0
    log(f"generated {len(graphs)} graphs in {gen_s:.1f} s")
    B.build()
    K.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    Gs = [K.Graph.from_inputs(g, skip_validate=True) for g in graphs]
    Qs = [K.Query(G, eps=0.02, delta=0.1, seed=1000 + i) for i, G in enumerate(Gs)]
    cost = [AT.estimated_cost(q) for q in Qs]
    by_cost = sorted(range(len(Qs)), key=lambda i: cost[i])
    Qsjf = [Qs[i] for i in by_cost]              # shortest expected work first
    max_n = max(g.n for g in graphs)
    pool = AT.BatchPool(max_n)
    tune = {}
    if args.autotune:
        best_b, trials, tune_s = AT.autotune(Qs, pool, log=log)
        tune["batched"] = {"seconds": tune_s, "trials": [dict(dataclasses.asdict(s), ms=ms) for s, ms in trials]}
        best_e, trials, tune_s = AT.autotune(Qsjf, pool, log=log, runner=AT.run_each)
        tune["one_query_per_launch"] = {"seconds": tune_s,
                                        "trials": [dict(dataclasses.asdict(s), ms=ms) for s, ms in trials]}
    else:
        best_b = best_e = AT.Schedule(threads=args.threads, divisor=args.divisor, frames=args.frames)
    for t in list(pool.batches):
        if t not in (best_b.threads, best_e.threads):
            pool.batches.pop(t).free()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    log(f"schedules: batched {best_b}, one query per launch {best_e}")

    def batched(policy, queries):
        def fn():
            b = pool.get(best_b.threads)
            b.set_policy(policy)
            flush.fill_(1)
            r = AT.run_mix(b, queries, best_b)
            b.set_policy(K.Batch.ROUND_ROBIN)
            return r
        return fn

    def per_query():
        flush.fill_(1)
        return AT.run_each(pool.get(best_e.threads), Qsjf, best_e)

    def graph_epochs():
        flush.fill_(1)
        lens = [best_e.epoch_len(q.info().omega_ceil) for q in Qsjf]
        for q in Qsjf:
            q.reset()
        t_sub = K.device_clock()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for q, E in zip(Qsjf, lens):
            q.run_graph(E, epochs_per_graph=args.graph_epochs)
        e1.record(stream)
        e1.synchronize()
        infos = [q.info() for q in Qsjf]
        return {"ms": e0.elapsed_time(e1), "tts_ms": [(i.stop_ns - t_sub) / 1e6 for i in infos],
                "tau": [i.tau for i in infos], "stop_epoch": [i.stop_epoch for i in infos],
                "stopped": [i.stopped for i in infos]}

    def digest(queries, r):
        """Results in query-index order (tau, stop epoch, counters)."""
        pos = {id(q): k for k, q in enumerate(queries)}
        h = hashlib.sha256()
        for q in Qs:
            k = pos[id(q)]
            h.update(f"{r['tau'][k]},{r['stop_epoch'][k]};".encode())
            h.update(q.result(btilde=False)["counts"].tobytes())
        return h.hexdigest()[:16]

    # (name, runner, query order, schedule)
    forms = [("batched", batched(K.Batch.ROUND_ROBIN, Qs), Qs, best_b),
             ("batched_shortest_first", batched(K.Batch.IN_ORDER, Qsjf), Qsjf, best_b),
             ("one_query_per_launch", per_query, Qsjf, best_e),
             ("graph_epochs", graph_epochs, Qsjf, best_e)]
    out, digests, clk_all = {}, {}, []
    for name, fn, order, sched in forms:
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        clocks = ClockSampler(local_rank)
        clocks.start()
        runs = [fn() for _ in range(args.steps)]
        torch.cuda.synchronize()
        clk_all.append(clocks.stop())
        for r in runs:
            assert all(r["stopped"]), f"{name}: a query did not stop"
        d = digest(order, runs[-1])
        digests.setdefault(sched, d)
        assert digests[sched] == d, f"{name}: results differ from the other form with the same schedule"
        ms = statistics.mean(r["ms"] for r in runs)
        out[name] = tts_summary(ms, sum(runs[-1]["tau"]), runs[-1]["tts_ms"])
        out[name]["schedule"] = dataclasses.asdict(sched)
        out[name]["samples"] = sum(runs[-1]["tau"])
        if "alone_ms" in runs[-1]:
            out[name]["alone_p50_ms"] = percentile(runs[-1]["alone_ms"], 50)
        log(name, json.dumps(out[name]))
    clk = next((c for c in clk_all if c), None)
    b = out["batched"]
    line = {
        "metric": "shortest-path samples/sec and time-to-(eps,delta) stop over a mix of queries",
        "value": b["samples_per_s"], "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["makespan_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": BATCHED_DESC, "queries": len(Qs), "n_total": sum(g.n for g in graphs),
                   "nnz_total": sum(g.nnz for g in graphs), "max_n": max_n,
                   "l2": "flushed before every step (256 MiB write); adjacency total far above L2",
                   "generation_s": gen_s},
        "samples_per_step": b["samples"],
        "forms": out,
        "speedup_vs_one_query_per_launch": out["one_query_per_launch"]["makespan_ms"] / b["makespan_ms"],
        "speedup_vs_graph_epochs": out["graph_epochs"]["makespan_ms"] / b["makespan_ms"],
        "results_identical_within_schedule": True,
        "autotune": tune or None,
        "gpu_launches": args.steps,          # the batched form: one persistent launch per timed step
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving: a Poisson stream of queries, continuous batching vs one at a time
# ---------------------------------------------------------------------------

def run_serve(args, local_rank):
    import torch

    from paper_1910_11039_gb300 import build as B
    from paper_1910_11039_gb300 import inputs
    from paper_1910_11039_gb300 import kadabra as K
    from paper_1910_11039_gb300.autotune import Schedule
    from paper_1910_11039_gb300.server import Request, Server

    if args.serve_pool == "full":
        pool = list(inputs.SERVING_POOL)
    elif args.serve_pool == "mixed":
        pool = [f"rmat{s}" for s in range(14, 21)] + ["grid1024"]
    else:
        pool = [k for k in inputs.SERVING_POOL if k.startswith("rmat")]
    reqs = inputs.serving_requests(count=args.serve_queries, rate=args.serve_rate, pool=pool)
    used = sorted({r["graph"] for r in reqs})
    t0 = time.perf_counter()
    host_graphs = {k: inputs.graph_from_spec(inputs.SERVING_POOL[k], k) for k in used}
    gen_s = time.perf_counter() - t0
    log(f"generated {len(used)} graphs in {gen_s:.1f} s")
    B.build()
    K.load()
    torch.cuda.set_device(local_rank)
    sched = Schedule(threads=args.threads, divisor=args.divisor, frames=args.frames)
    srv = Server(host_graphs, schedule=sched, step_ms=args.step_ms, policy=args.serve_policy,
                 keep_results=False)
    del host_graphs
    # warm-up: a few requests of the stream, served at once and discarded
    warm = [Request(**dict(r, arrival=0.0)) for r in reqs[:max(8, 4 * args.warmup)]]
    srv.run(warm, realtime=False)
    srv.run_one_at_a_time([Request(**dict(r, arrival=0.0)) for r in reqs[:4]], realtime=False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    clocks.start()
    done = srv.run([Request(**r) for r in reqs])
    clk = clocks.stop()
    s_batched = srv.summary(done)
    log("continuous batching", json.dumps(s_batched))
    done1 = srv.run_one_at_a_time([Request(**r) for r in reqs])
    s_plain = srv.summary(done1)
    log("one at a time", json.dumps(s_plain))
    a = {r.rid: (r.tau, r.stop_epoch) for r in done}
    b = {r.rid: (r.tau, r.stop_epoch) for r in done1}
    same = sum(1 for k in a if a[k] == b.get(k))
    line = {
        "metric": "time-to-(eps,delta) stop p50/p99 and samples/sec under a Poisson query stream",
        "value": s_batched["samples_per_s"], "unit": "samples/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * s_batched["wall_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"Poisson stream, rate {args.serve_rate}/s, {args.serve_queries} queries, graphs "
                               f"uniform over {pool}, eps uniform over {{0.01, 0.005}}, delta 0.1, stream seed 5",
                   "pool": args.serve_pool, "graphs_used": used, "schedule": dataclasses.asdict(sched),
                   "step_ms": args.step_ms, "policy": args.serve_policy, "generation_s": gen_s},
        "tts_p50_s": s_batched["tts_p50_s"], "tts_p99_s": s_batched["tts_p99_s"],
        "continuous_batching": s_batched,
        "one_query_at_a_time": s_plain,
        "results_identical": {"compared": len(a), "same_tau_and_stop_epoch": same},
        "gpu_launches": s_batched["steps"],
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: per workload, 20 for rmat20)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="rmat26", choices=list(WORKLOADS))
    ap.add_argument("--epoch", type=int, default=1024)
    ap.add_argument("--mode", default="pipelined", choices=["pipelined", "epochs", "batched", "serve", "sharded"],
                    help="pipelined/epochs: one query on --workload; sharded: one query split over the ranks; "
                         "batched: 64 queries of uneven size; serve: a Poisson stream of queries")
    ap.add_argument("--serve-queries", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-pool", default="rmat", choices=["rmat", "full", "mixed"],
                    help="rmat: R-MAT scale 14-24; full: also the perturbed grids 1024^2-4096^2; "
                         "mixed: R-MAT scale 14-20 and the 1024^2 grid")
    ap.add_argument("--serve-policy", default="fifo", choices=["fifo", "shortest", "round_robin"])
    ap.add_argument("--step-ms", type=float, default=20.0, help="serve mode: target length of a batch step")
    ap.add_argument("--autotune", action="store_true", help="batched mode: search the schedule first")
    ap.add_argument("--divisor", type=int, default=32, help="batched mode: epoch length = omega / divisor")
    ap.add_argument("--graph-epochs", type=int, default=4, help="epochs per CUDA graph (graph_epochs form)")
    ap.add_argument("--frames", type=int, default=None,
                    help="epoch frames in flight (default: 12 for one pipelined query, 8 for batched/serve schedules)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--slots", type=int, default=0, help="samples in flight (0 = fill the GPU)")
    ap.add_argument("--threads", type=int, default=None, help="threads per sampling CTA (default: per workload)")
    ap.add_argument("--cpu-samples", type=int, default=None,
                    help="oracle samples for the CPU baseline (split over host cores)")
    ap.add_argument("--ref-samples", type=int, default=None, help="oracle samples per reference step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-oracle-stop", action="store_true", help="skip the oracle's own run to the stop")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference" or os.environ.get("KADABRA_BENCH_ALLOW_SHORT"), \
        "at least 3 warm-up steps"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    # defaults sized so that each workload's run ends within minutes
    if args.mode in ("batched", "serve"):
        if args.steps is None:
            args.steps = 2
        if args.threads is None:
            args.threads = 1024
    if args.frames is None:
        # one pipelined query: 12 frames (R-MAT-26 median time to stop 9.8 ms against 11.1 ms
        # with 8, same with 16; R-MAT-20 alike); the many-query schedules keep 8
        args.frames = 12 if args.mode == "pipelined" else 8
    for key, default in (("steps", 20), ("e2e_steps", 3), ("cpu_samples", 48000), ("ref_samples", 16000),
                         ("threads", 1024)):
        if getattr(args, key) is None:
            setattr(args, key, wl.get(key, default))
    if args.mode in ("batched", "serve"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": f"the {args.mode} mode has no CPU form; the "
                              "oracle arm runs on the single-query workloads"}), flush=True)
            return
        if rank == 0:
            (run_batched if args.mode == "batched" else run_serve)(args, local_rank)
        return

    from paper_1910_11039_gb300 import inputs
    g = inputs.config_graph(wl["graph"])

    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        run_reference(args, wl, g, rank, world)
        return

    # CPU baseline first: the oracle runs on host threads before any CUDA call
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu and args.mode != "sharded":
        cpu_baseline = cpu_baseline_for(g, wl, args)
    if args.mode == "sharded":
        import torch
        torch.cuda.set_device(local_rank)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        torch.distributed.init_process_group("nccl", rank=rank, world_size=world)
        try:
            run_sharded(args, wl, g, rank, world, local_rank)
        finally:
            torch.distributed.destroy_process_group()
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_gpu(args, wl, g, rank, world, local_rank, cpu_baseline)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
