"""Continuous-batching betweenness server on one GPU.

Requests (graph, eps, delta, seed) arrive over time.  The server keeps the
graphs resident and runs every admitted query inside one shared persistent
launch per step (kadabra_batch_step with a sample budget, so a step lasts
about `step_ms`).  Between steps it

  * admits arrived requests while their device state fits the memory budget
    (query state: counters, budgets, calibration counts, epoch logs; the
    graphs and the batch's sampling scratch are reserved up front),
  * starts each new query's calibration samples, which then run in the next
    steps beside the other queries' adaptive samples (the paper's phase 2,
    Section III-A, done inside the batch),
  * turns a query whose calibration completed into an adaptive query
    (budgets on the host, epoch logs on the device),
  * retires queries whose stopping condition held (or that reached omega),
    reading their counters and freeing their state.

A query's state stays on the device for its whole life; its samples are
indexed by (seed, stream tag, sample index), so its result does not depend
on what else shares the launch: the same request alone and in any mix gives
the same tau, stop epoch and counters.

Time-to-stop is measured on the device clock: the stop check records the
global timer when it decides the stop, and the server maps that timer onto
the run's host clock once at start.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np

from . import kadabra as K
from .autotune import Schedule


@dataclasses.dataclass
class Request:
    rid: int
    graph: str
    eps: float
    delta: float = 0.1
    seed: int = 1
    arrival: float = 0.0          # seconds after the start of the run
    # filled in by the server
    admitted: float | None = None  # host time of admission (run clock)
    calibrated: float | None = None
    seen_done: float | None = None  # host time the completion was observed
    stop_time: float | None = None  # device time of the stop decision (run clock)
    tau: int = 0
    stop_epoch: int = -1
    epoch_len: int = 0
    omega_ceil: int = 0
    device_bytes: int = 0
    counts: np.ndarray | None = None

    @property
    def time_to_stop(self) -> float | None:
        return None if self.stop_time is None else self.stop_time - self.arrival


class _Active:
    __slots__ = ("req", "q", "phase", "bytes", "n_calib")

    def __init__(self, req, q, nbytes, n_calib):
        self.req, self.q, self.phase, self.bytes, self.n_calib = req, q, 1, nbytes, n_calib


class Server:
    """policy "fifo": earlier arrivals take samples first (the batch's
    IN_ORDER policy over the active list in arrival order); "shortest": the
    query with the least expected work left goes first (IN_ORDER over the
    active list sorted by samples left times graph size, a proxy for the cost
    of a sample); "round_robin": every active query takes samples at the same
    rate."""

    def __init__(self, graphs: dict, threads: int = 1024, slots: int = 0, schedule: Schedule | None = None,
                 memory_budget: int | None = None, step_ms: float = 20.0, policy: str = "fifo",
                 keep_results: bool = True, log=None):
        self.graphs = {}
        for key, g in graphs.items():
            self.graphs[key] = g if isinstance(g, K.Graph) else K.Graph.from_inputs(g, skip_validate=True)
        infos = {k: G.info() for k, G in self.graphs.items()}
        off64 = {bool(i["offsets_64"]) for i in infos.values()}
        if len(off64) > 1:
            raise ValueError("all graphs of a server must use the same offset width")
        self.n = {k: int(i["n"]) for k, i in infos.items()}
        self.max_n = max(self.n.values())
        self.schedule = schedule or Schedule(threads=threads)
        self.batch = K.Batch(self.max_n, slots=slots, threads=self.schedule.threads,
                             offsets_64=off64.pop() if off64 else False)
        # a step hands out at least this many samples per slot, so that the
        # samples still running when the budget is spent (one per slot) are a
        # small share of it; long samples (high-diameter graphs) get more
        self.slots = int(self.batch.info()["slots"]) if hasattr(self.batch, "info") else 32
        self.min_budget = 8 * self.slots
        self.min_budget_long = 32 * self.slots
        if policy not in ("fifo", "shortest", "round_robin"):
            raise ValueError("policy must be 'fifo', 'shortest' or 'round_robin'")
        self.policy = policy
        self.batch.set_policy(K.Batch.ROUND_ROBIN if policy == "round_robin" else K.Batch.IN_ORDER)
        if memory_budget is None:
            import torch

            torch.cuda.synchronize()
            free, _ = torch.cuda.mem_get_info()
            memory_budget = int(0.8 * free)
        self.memory_budget = int(memory_budget)
        self.step_ms = step_ms
        self.keep_results = keep_results
        self.log = log
        self.used = 0
        self.vd: dict[str, int] = {}      # vertex-diameter bound per graph, computed by its first query
        self.stats = {"steps": 0, "step_ms": 0.0, "samples": 0, "cal_samples": 0, "admit_waits": 0,
                      "max_active": 0, "peak_bytes": 0}

    # -- helpers -----------------------------------------------------------

    def _state_bytes_estimate(self, key: str) -> int:
        """Device bytes of a query before its epoch logs are known."""
        return 40 * self.n[key] + (1 << 20)

    def _create(self, r: "Request"):
        """Phase 1 of a request's query (the graph's vertex-diameter bound is
        computed once, by its first query, and reused)."""
        q = K.Query(self.graphs[r.graph], calibrate=False, eps=r.eps, delta=r.delta, seed=r.seed,
                    threads=self.schedule.threads, vertex_diameter=self.vd.get(r.graph, 0))
        if r.graph not in self.vd:
            self.vd[r.graph] = int(q.info().vertex_diameter)
        return q

    def _work_left(self, a: "_Active") -> float:
        """Expected work of an active query: samples it may still take (its
        calibration samples, or omega, as an upper bound known without a
        device read) times its graph's vertex count."""
        left = a.n_calib if a.phase == 1 else a.req.omega_ceil
        return float(left) * self.n[a.req.graph]

    def _log_bytes(self, vd: int, E: int) -> int:
        return 4 * self.schedule.frames * E * max(1, vd - 2)

    def close(self):
        self.batch.free()
        for G in self.graphs.values():
            G.free()
        self.graphs = {}

    # -- the loop ----------------------------------------------------------

    def run(self, requests, realtime: bool = True, clock=time.perf_counter):
        """Serve `requests` (any order; each has an arrival time in seconds).
        With realtime=False every request is taken as already arrived.
        Returns the requests with their results and timings."""
        self.stats = {"steps": 0, "step_ms": 0.0, "samples": 0, "cal_samples": 0, "admit_waits": 0,
                      "max_active": 0, "peak_bytes": 0, "tau": 0}
        future = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        pending: deque[Request] = deque()
        active: list[_Active] = []
        done: list[Request] = []
        budget = 4096
        t0 = clock()
        dev0 = K.device_clock()
        t_dev = clock()
        t0 = 0.5 * (t0 + t_dev)          # host time matching dev0

        def now():
            return clock() - t0

        while future or pending or active:
            t = now()
            while future and (not realtime or future[0].arrival <= t):
                pending.append(future.popleft())
            # admission by device memory
            while pending:
                r = pending[0]
                est = self._state_bytes_estimate(r.graph)
                if active and self.used + est > self.memory_budget:
                    self.stats["admit_waits"] += 1
                    break
                pending.popleft()
                q = self._create(r)
                inf = q.info()
                r.omega_ceil = int(inf.omega_ceil)
                r.epoch_len = self.schedule.epoch_len(r.omega_ceil)
                nbytes = int(inf.device_bytes) + self._log_bytes(int(inf.vertex_diameter), r.epoch_len)
                r.device_bytes = nbytes
                self.used += nbytes
                q.calibration_begin()
                r.admitted = now()
                active.append(_Active(r, q, nbytes, int(inf.n_calib)))
            self.stats["max_active"] = max(self.stats["max_active"], len(active))
            self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.used)
            if not active:
                if future and realtime:
                    time.sleep(max(0.0, min(0.05, future[0].arrival - now())))
                continue
            # one step over every active query (list order = priority under IN_ORDER)
            if self.policy == "shortest":
                active.sort(key=self._work_left)
            self.batch.step([a.q for a in active], sample_budget=budget)
            ms = self.batch.last_ms()
            self.stats["steps"] += 1
            self.stats["step_ms"] += ms
            floor = self.min_budget_long if any(self.vd.get(a.req.graph, 0) > 64 for a in active) else self.min_budget
            budget = int(min(1 << 22, max(floor, budget * self.step_ms / max(ms, 1e-3))))
            states = self.batch.poll(len(active))
            still = []
            for a, state in zip(active, states):
                if a.phase == 1:
                    if state == 1:
                        a.q.calibration_finish()
                        a.q.pipeline_begin(a.req.epoch_len, frames=self.schedule.frames)
                        a.phase = 2
                        a.req.calibrated = now()
                    still.append(a)
                    continue
                if state != 2:
                    still.append(a)
                    continue
                inf = a.q.info()
                self.stats["cal_samples"] += int(inf.n_calib)
                r = a.req
                r.seen_done = now()
                r.stop_time = (int(inf.stop_ns) - dev0) / 1e9
                r.tau = int(inf.tau)
                r.stop_epoch = int(inf.stop_epoch)
                self.stats["samples"] += int(inf.samples)
                self.stats["tau"] += r.tau
                if self.keep_results:
                    r.counts = a.q.result(btilde=False)["counts"]
                a.q.free()
                self.used -= a.bytes
                done.append(r)
            active = still
        self.stats["wall_s"] = now()
        return done

    def run_one_at_a_time(self, requests, realtime: bool = True, clock=time.perf_counter):
        """The same stream served the plain way: one query at a time in
        arrival order, its calibration in one launch and its adaptive phase
        in one more launch (same kernels, scratch and schedule, no sharing)."""
        future = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        done: list[Request] = []
        self.batch.set_policy(K.Batch.IN_ORDER)
        t0 = clock()
        dev0 = K.device_clock()
        t0 = 0.5 * (t0 + clock())
        steps, step_ms, samples, cal = 0, 0.0, 0, 0

        def now():
            return clock() - t0

        while future:
            r = future.popleft()
            if realtime and r.arrival > now():
                time.sleep(r.arrival - now())
            q = self._create(r)
            r.admitted = now()
            inf = q.info()
            r.omega_ceil = int(inf.omega_ceil)
            r.epoch_len = self.schedule.epoch_len(r.omega_ceil)
            q.calibration_begin()
            self.batch.step([q])
            step_ms += self.batch.last_ms()
            q.calibration_finish()
            r.calibrated = now()
            q.pipeline_begin(r.epoch_len, frames=self.schedule.frames)
            self.batch.step([q])
            step_ms += self.batch.last_ms()
            steps += 2
            inf = q.info()
            r.seen_done = now()
            r.stop_time = (int(inf.stop_ns) - dev0) / 1e9
            r.tau, r.stop_epoch = int(inf.tau), int(inf.stop_epoch)
            samples += int(inf.samples)
            cal += int(inf.n_calib)
            if self.keep_results:
                r.counts = q.result(btilde=False)["counts"]
            q.free()
            done.append(r)
        self.batch.set_policy(K.Batch.ROUND_ROBIN if self.policy == "round_robin" else K.Batch.IN_ORDER)
        self.stats.update(steps=steps, step_ms=step_ms, samples=samples, cal_samples=cal, wall_s=now(),
                          tau=sum(r.tau for r in done), max_active=1, peak_bytes=0, admit_waits=0)
        return done

    def summary(self, done) -> dict:
        tts = sorted(r.time_to_stop for r in done)
        wall = self.stats["wall_s"]
        pct = lambda p: tts[min(len(tts) - 1, max(0, int(round(p / 100.0 * (len(tts) - 1)))))] if tts else None
        return {"queries": len(done), "tts_p50_s": pct(50), "tts_p99_s": pct(99), "tts_max_s": tts[-1] if tts else None,
                "samples": self.stats["samples"], "cal_samples": self.stats["cal_samples"],
                "tau_total": self.stats.get("tau", 0),
                "samples_per_s": (self.stats["samples"] + self.stats["cal_samples"]) / wall if wall else None,
                "adaptive_samples_per_s": self.stats["samples"] / wall if wall else None,
                "wall_s": wall, "steps": self.stats["steps"],
                "gpu_busy_frac": self.stats["step_ms"] / 1e3 / wall if wall else None,
                "max_active": self.stats["max_active"], "peak_state_bytes": self.stats["peak_bytes"],
                "admission_waits": self.stats["admit_waits"], "memory_budget": self.memory_budget}
