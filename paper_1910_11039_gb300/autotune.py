"""Schedule autotuner for many queries sharing one persistent launch.

The paper tunes one knob of its epoch framework, the number of samples
between aggregations (Section IV-C: n0 as a function of processes and
threads).  On one GPU the knobs that decide how fast a mix of queries reaches
its stopping condition are:

  threads  threads per sampling CTA, i.e. warps per in-flight sample
           (128 .. 1024 = 4 .. 32 warps).  Fewer warps per sample put more
           samples in flight per SM, which pays on high-diameter graphs whose
           samples are long chains of small BFS layers; more warps per
           sample pay on low-diameter graphs with wide layers.
  epoch    each query's epoch length E = omega / divisor, rounded to a power
           of two and clamped.  Short epochs stop closer to the first epoch
           at which the condition holds (at most one epoch of samples beyond
           it is taken); long epochs check less often.
  frames   epochs in flight per query (epoch logs).  More frames let more
           CTAs work on the same query while its oldest epoch waits for its
           check, at the price of more samples beyond the stopping epoch.

A trial runs the whole mix to its stop in one batch step and then restarts
the queries (their calibration is kept).  The result of every query depends
only on its epoch length, so a trial is a real run and its makespan is the
quantity being minimised.  Search order: threads at the default divisor and
frames, then the divisor, then frames (coordinate descent, one pass).
"""
from __future__ import annotations

import dataclasses
import math
import time

from . import kadabra as K


@dataclasses.dataclass(frozen=True)
class Schedule:
    threads: int = 1024
    divisor: int = 32
    frames: int = 8
    min_epoch: int = 32
    max_epoch: int = 4096

    def epoch_len(self, omega_ceil: int) -> int:
        """Power of two nearest omega / divisor, clamped to [min_epoch, max_epoch]."""
        x = max(1.0, omega_ceil / self.divisor)
        e = 1 << max(0, round(math.log2(x)))
        return int(min(self.max_epoch, max(self.min_epoch, e)))


def begin_all(queries, schedule: Schedule, stream=None, reset=True):
    """Restart each query's adaptive phase and begin its pipeline with the
    schedule's epoch length and frames.  Returns the epoch lengths."""
    lens = []
    for q in queries:
        if reset:
            q.reset(stream)
        E = schedule.epoch_len(q.info().omega_ceil)
        q.pipeline_begin(E, frames=schedule.frames, stream=stream)
        lens.append(E)
    return lens


def run_mix(batch: "K.Batch", queries, schedule: Schedule, stream=None) -> dict:
    """Run every query to its stop in one persistent launch.  Returns the
    launch's device time, each query's device time-to-stop measured from the
    launch's submission, tau and stop epoch."""
    lens = begin_all(queries, schedule, stream)
    t0 = K.device_clock(stream)
    batch.step(queries, stream=stream)
    ms = batch.last_ms()
    infos = [q.info() for q in queries]
    return {"ms": ms, "epoch_lens": lens,
            "tts_ms": [(i.stop_ns - t0) / 1e6 if i.stopped else float("nan") for i in infos],
            "tau": [i.tau for i in infos], "stop_epoch": [i.stop_epoch for i in infos],
            "stopped": [i.stopped for i in infos]}


def run_each(batch: "K.Batch", queries, schedule: Schedule, stream=None) -> dict:
    """The same queries one launch each, back to back on one stream (no host
    synchronisation between them).  Time-to-stop is measured from the
    submission of the first launch."""
    import torch

    lens = begin_all(queries, schedule, stream)
    t0 = K.device_clock(stream)
    st = torch.cuda.current_stream() if stream is None else stream
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(queries) + 1)]
    evs[0].record(st)
    for k, q in enumerate(queries):
        batch.step([q], stream=stream)
        evs[k + 1].record(st)
    evs[-1].synchronize()
    infos = [q.info() for q in queries]
    return {"ms": evs[0].elapsed_time(evs[-1]), "epoch_lens": lens,
            "alone_ms": [evs[k].elapsed_time(evs[k + 1]) for k in range(len(queries))],
            "tts_ms": [(i.stop_ns - t0) / 1e6 if i.stopped else float("nan") for i in infos],
            "tau": [i.tau for i in infos], "stop_epoch": [i.stop_epoch for i in infos],
            "stopped": [i.stopped for i in infos]}


def estimated_cost(q) -> float:
    """Expected device time of a query alone (ms): omega times the mean time
    per sample of its oldest logged sampling launch (the calibration launch,
    when called before any other launch of the query)."""
    log = [ls for ls in q.launch_log(256) if ls.samples > 0]
    per = log[0].ms / log[0].samples if log else 1.0
    return q.info().omega_ceil * per


class BatchPool:
    """One kadabra Batch per thread count, created on first use."""

    def __init__(self, max_n: int, offsets_64: bool = False):
        self.max_n = max_n
        self.off64 = offsets_64
        self.batches: dict[int, K.Batch] = {}

    def get(self, threads: int) -> "K.Batch":
        if threads not in self.batches:
            self.batches[threads] = K.Batch(self.max_n, threads=threads, offsets_64=self.off64)
        return self.batches[threads]

    def keep_only(self, threads: int):
        for t in list(self.batches):
            if t != threads:
                self.batches.pop(t).free()


def autotune(queries, pool: BatchPool, threads=(128, 256, 512, 1024), divisors=(8, 16, 32, 64, 128),
             frames=(4, 8, 16), base: Schedule | None = None, stream=None, log=None, runner=run_mix):
    """Coordinate-descent search over (threads, divisor, frames) for the form
    `runner` (run_mix: all queries in one launch; run_each: one launch per
    query).  Returns (best schedule, list of trials (schedule, makespan ms),
    seconds spent)."""
    base = base or Schedule()
    trials = []
    seen: dict[Schedule, float] = {}
    t_start = time.perf_counter()

    def trial(s: Schedule) -> float:
        if s in seen:
            return seen[s]
        r = runner(pool.get(s.threads), queries, s, stream)
        ms = r["ms"] if all(r["stopped"]) else float("inf")
        seen[s] = ms
        trials.append((s, ms))
        if log:
            log(f"autotune threads={s.threads} divisor={s.divisor} frames={s.frames}: {ms:.2f} ms")
        return ms

    best = base
    best_ms = trial(best)
    for field, values in (("threads", threads), ("divisor", divisors), ("frames", frames)):
        for v in values:
            s = dataclasses.replace(best, **{field: v})
            ms = trial(s)
            if ms < best_ms:
                best, best_ms = s, ms
    return best, trials, time.perf_counter() - t_start
