"""CPU oracle for KADABRA adaptive-sampling betweenness (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg, never by the library.  The arithmetic lives
in ``kadabra_oracle.c`` (plain C, built with ``-ffp-contract=off``); this
module only builds it with gcc and marshals numpy arrays through ctypes.

Parity status of each function (details in the C file's header):
  philox4x64_10, brandes, sample_pair / sample / run_samples,
  vertex_diameter_*            pinned (numpy Philox, networkx, closed forms,
                               path enumeration)
  omega, calibrate_L, stop_functions, check_stop, kadabra
                               the paper does not print these formulas (read
                               from KADABRA's publication); pinned by hand
                               values (omega), closed-form and 50-digit roots
                               (balanced rule, f and g), Table II sample
                               counts <= omega and the epsilon guarantee
                               against Brandes
  kadabra_threads              the same phases as kadabra, each phase's
                               sample indices split over host threads and
                               the per-thread counters summed
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kadabra_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


class SampleInfo(C.Structure):
    _fields_ = [("s", C.c_int64), ("t", C.c_int64), ("d", C.c_int64),
                ("sigma_lo", C.c_uint64), ("sigma_hi", C.c_uint64),
                ("meet_size", C.c_int64), ("chosen", C.c_int64),
                ("e_scan", C.c_int64), ("n_interior", C.c_int64),
                ("scaled", C.c_int32), ("overflow", C.c_int32)]

    @property
    def sigma(self) -> int:
        return (int(self.sigma_hi) << 64) | int(self.sigma_lo)


class RunStats(C.Structure):
    _fields_ = [("samples", C.c_int64), ("e_scan", C.c_int64), ("connected", C.c_int64),
                ("interior", C.c_int64), ("scaled", C.c_int64), ("overflow", C.c_int64)]


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("delta", C.c_double), ("seed", C.c_uint64),
                ("vertex_diameter", C.c_int64), ("n_calib", C.c_int64),
                ("epoch_len", C.c_int64), ("delta_rule", C.c_int32), ("strict", C.c_int32),
                ("beta", C.c_double), ("max_epochs", C.c_int64)]


class Result(C.Structure):
    _fields_ = [("omega", C.c_double), ("vd", C.c_int64), ("n_calib", C.c_int64),
                ("K", C.c_int32), ("stopped", C.c_int32), ("tau", C.c_uint64),
                ("epochs", C.c_int64), ("stop_epoch", C.c_int64),
                ("max_f", C.c_double), ("max_g", C.c_double), ("C", C.c_double),
                ("e_scan", C.c_int64), ("overflow", C.c_int64)]


_P = C.c_void_p
_I64 = C.c_int64
_U64 = C.c_uint64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_philox4x64_10.argtypes = [_P, _P, _P]
            L.orc_sigma_bits.argtypes = [_I64, _I64]
            L.orc_sigma_bits.restype = C.c_int
            L.orc_ws_create.argtypes = [_I64]
            L.orc_ws_create.restype = _P
            L.orc_ws_free.argtypes = [_P]
            L.orc_sample_pair.argtypes = [_I64, _P, _P, _P, _I64, _I64, _U64, _U64, _U64,
                                          C.c_int, C.c_int, _P, C.POINTER(SampleInfo)]
            L.orc_sample_pair.restype = _I64
            L.orc_sample.argtypes = [_I64, _P, _P, _P, _U64, _U64, _U64, C.c_int, C.c_int,
                                     _P, C.POINTER(SampleInfo)]
            L.orc_sample.restype = _I64
            L.orc_draw_pair.argtypes = [_I64, _U64, _U64, _U64, C.POINTER(_I64), C.POINTER(_I64)]
            L.orc_run_samples.argtypes = [_I64, _P, _P, _U64, _U64, _U64, _U64, C.c_int, C.c_int,
                                          _P, C.POINTER(RunStats)]
            L.orc_run_samples.restype = _I64
            L.orc_run_samples_ws.argtypes = [_I64, _P, _P, _P, _P, _U64, _U64, _U64, _U64, C.c_int, C.c_int,
                                             _P, C.POINTER(RunStats)]
            L.orc_run_samples_ws.restype = _I64
            L.orc_vertex_diameter_bound.argtypes = [_I64, _P, _P]
            L.orc_vertex_diameter_bound.restype = _I64
            L.orc_vertex_diameter_exact.argtypes = [_I64, _P, _P]
            L.orc_vertex_diameter_exact.restype = _I64
            L.orc_omega.argtypes = [C.c_double, C.c_double, _I64]
            L.orc_omega.restype = C.c_double
            L.orc_calibrate_L.argtypes = [_I64, _P, _I64, C.c_double, C.c_double, C.c_int,
                                          C.c_double, _P, _P, C.POINTER(C.c_double)]
            L.orc_stop_functions.argtypes = [C.c_uint32, _U64, C.c_double, C.c_double, C.c_double,
                                             C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_check_stop.argtypes = [_I64, _P, _U64, C.c_double, C.c_double, _P, _P,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_check_stop.restype = C.c_int
            L.orc_kadabra.argtypes = [_I64, _P, _P, C.POINTER(Params), _P, _P, _P, _P,
                                      C.POINTER(Result)]
            L.orc_kadabra.restype = C.c_int
            L.orc_brandes.argtypes = [_I64, _P, _P, _P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    return off, col


def philox4x64_10(ctr, key) -> list[int]:
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(x) for x in out]


def sigma_bits(n: int, max_degree: int) -> int:
    return lib().orc_sigma_bits(n, max_degree)


def graph_sigma_bits(g) -> int:
    return sigma_bits(g.n, g.max_degree)


class Workspace:
    """Reusable per-thread scratch for single samples."""

    def __init__(self, g):
        self.g = g
        self.off, self.col = _csr(g)
        self.ws = lib().orc_ws_create(g.n)
        self.path = np.zeros(max(g.n, 1), dtype=np.int32)
        self.K = graph_sigma_bits(g)

    def __del__(self):
        try:
            lib().orc_ws_free(self.ws)
        except Exception:
            pass

    def sample_pair(self, s, t, seed, tag, idx, strict=False, K=None):
        info = SampleInfo()
        np_ = lib().orc_sample_pair(self.g.n, _ptr(self.off), _ptr(self.col), self.ws, s, t,
                                    seed, tag, idx, self.K if K is None else K, int(strict),
                                    _ptr(self.path), C.byref(info))
        return self.path[:np_].copy(), info

    def run_samples(self, seed, tag, begin, end, counts=None, strict=False, K=None):
        """counts[x] += #samples in [begin, end) with x interior, reusing this
        workspace; returns (counts, RunStats)."""
        if counts is None:
            counts = np.zeros(self.g.n, dtype=np.uint32)
        st = RunStats()
        lib().orc_run_samples_ws(self.g.n, _ptr(self.off), _ptr(self.col), self.ws, _ptr(self.path), seed, tag,
                                 begin, end, self.K if K is None else K, int(strict), _ptr(counts), C.byref(st))
        return counts, st

    def sample(self, seed, tag, idx, strict=False, K=None):
        info = SampleInfo()
        np_ = lib().orc_sample(self.g.n, _ptr(self.off), _ptr(self.col), self.ws,
                               seed, tag, idx, self.K if K is None else K, int(strict),
                               _ptr(self.path), C.byref(info))
        return self.path[:np_].copy(), info


def draw_pair(n, seed, tag, idx):
    s, t = _I64(), _I64()
    lib().orc_draw_pair(n, seed, tag, idx, C.byref(s), C.byref(t))
    return s.value, t.value


def run_samples(g, seed, tag, begin, end, counts=None, strict=False, K=None):
    """counts[x] += #samples in [begin, end) whose path has x as interior vertex."""
    off, col = _csr(g)
    if counts is None:
        counts = np.zeros(g.n, dtype=np.uint32)
    st = RunStats()
    lib().orc_run_samples(g.n, _ptr(off), _ptr(col), seed, tag, begin, end,
                          graph_sigma_bits(g) if K is None else K, int(strict),
                          _ptr(counts), C.byref(st))
    return counts, st


def vertex_diameter_bound(g) -> int:
    off, col = _csr(g)
    return lib().orc_vertex_diameter_bound(g.n, _ptr(off), _ptr(col))


def vertex_diameter_exact(g) -> int:
    off, col = _csr(g)
    return lib().orc_vertex_diameter_exact(g.n, _ptr(off), _ptr(col))


def omega(eps, delta, vd) -> float:
    return lib().orc_omega(eps, delta, vd)


def calibrate_L(cal_counts, n_cal, eps, delta, rule=1, beta=1e-3):
    cal = np.ascontiguousarray(cal_counts, dtype=np.uint32)
    n = cal.shape[0]
    LL = np.zeros(n, dtype=np.float64)
    LU = np.zeros(n, dtype=np.float64)
    Cc = C.c_double()
    lib().orc_calibrate_L(n, _ptr(cal), n_cal, eps, delta, rule, beta, _ptr(LL), _ptr(LU),
                          C.byref(Cc))
    return LL, LU, Cc.value


def stop_functions(c, tau, omega_, LL, LU):
    f, g = C.c_double(), C.c_double()
    lib().orc_stop_functions(c, tau, omega_, LL, LU, C.byref(f), C.byref(g))
    return f.value, g.value


def check_stop(counts, tau, omega_, eps, LL, LU):
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    LL = np.ascontiguousarray(LL, dtype=np.float64)
    LU = np.ascontiguousarray(LU, dtype=np.float64)
    mf, mg = C.c_double(), C.c_double()
    stop = lib().orc_check_stop(counts.shape[0], _ptr(counts), tau, omega_, eps, _ptr(LL),
                                _ptr(LU), C.byref(mf), C.byref(mg))
    return bool(stop), mf.value, mg.value


def kadabra(g, eps, delta, seed=1, vertex_diameter=0, n_calib=0, epoch_len=1000,
            delta_rule=1, strict=False, beta=1e-3, max_epochs=1 << 40):
    """Run the whole method; returns (counts, cal_counts, L_L, L_U, Result)."""
    off, col = _csr(g)
    P = Params(eps, delta, seed, vertex_diameter, n_calib, epoch_len, delta_rule, int(strict),
               beta, max_epochs)
    counts = np.zeros(g.n, dtype=np.uint32)
    cal = np.zeros(g.n, dtype=np.uint32)
    LL = np.zeros(g.n, dtype=np.float64)
    LU = np.zeros(g.n, dtype=np.float64)
    R = Result()
    lib().orc_kadabra(g.n, _ptr(off), _ptr(col), C.byref(P), _ptr(counts), _ptr(cal), _ptr(LL),
                      _ptr(LU), C.byref(R))
    return counts, cal, LL, LU, R


def brandes(g) -> np.ndarray:
    """Exact normalised betweenness b(x) over ordered pairs (fp64)."""
    off, col = _csr(g)
    b = np.zeros(g.n, dtype=np.float64)
    lib().orc_brandes(g.n, _ptr(off), _ptr(col), _ptr(b))
    return b


def _split_run(g, seed, tag, begin, end, threads, K=None, strict=False, pool=None):
    """Samples [begin, end) of stream `tag` split into `threads` contiguous
    index ranges, each run on its own host thread (ctypes releases the GIL),
    on the workspaces of `pool` when given; returns the summed counters and
    the summed stats."""
    import concurrent.futures as cf
    if pool is not None:
        threads = len(pool)
    cuts = [begin + (end - begin) * k // threads for k in range(threads + 1)]

    def part(k):
        if pool is not None:
            return pool[k].run_samples(seed, tag, cuts[k], cuts[k + 1], K=K, strict=strict)
        return run_samples(g, seed, tag, cuts[k], cuts[k + 1], K=K, strict=strict)

    with cf.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(part, range(threads)))
    counts = np.zeros(g.n, dtype=np.uint32)
    tot = RunStats()
    for c, st in parts:
        counts += c
        for f, _ in RunStats._fields_:
            setattr(tot, f, getattr(tot, f) + getattr(st, f))
    return counts, tot


def kadabra_threads(g, eps, delta, seed=1, vertex_diameter=0, n_calib=0, epoch_len=1000, delta_rule=1,
                    strict=False, beta=1e-3, max_epochs=1 << 40, threads=None, on_epoch=None):
    """The whole method with every phase's samples spread over host threads:
    phase 1 diameter bound -> omega, phase 2 calibration samples (tag 0) ->
    L_L, L_U, phase 3 epochs of `epoch_len` adaptive samples (tag 1), each
    followed by the stop check on the snapshot of samples [0, tau)
    (Section III-A, III-B).  The same C functions, in the same order and with
    the same clipping at ceil(omega) as kadabra(); only the sample loop of
    each epoch is split into index ranges, and counters are integer sums, so
    the result equals kadabra()'s.  Returns (counts, cal, L_L, L_U, info)."""
    import time
    threads = threads or max(1, len(os.sched_getaffinity(0)))
    pool = [Workspace(g) for _ in range(threads)]
    t0 = time.perf_counter()
    K = graph_sigma_bits(g)
    vd = vertex_diameter if vertex_diameter > 0 else vertex_diameter_bound(g)
    om = omega(eps, delta, vd)
    om_ceil = math.ceil(om)
    nc = n_calib if n_calib > 0 else max(1000, math.ceil(om / 100.0))
    cal, _ = _split_run(g, seed, 0, 0, nc, threads, K=K, strict=strict, pool=pool)
    LL, LU, Cc = calibrate_L(cal, nc, eps, delta, rule=delta_rule, beta=beta)
    t1 = time.perf_counter()
    counts = np.zeros(g.n, dtype=np.uint32)
    tau, stop_epoch, e_scan, epochs = 0, -1, 0, 0
    mf = mg = math.inf
    for e in range(max_epochs):
        m = min(epoch_len, om_ceil - tau) if tau < om_ceil else 0
        if m > 0:
            c, st = _split_run(g, seed, 1, tau, tau + m, threads, K=K, strict=strict, pool=pool)
            counts += c
            e_scan += st.e_scan
        tau += m
        epochs = e + 1
        stop, mf, mg = check_stop(counts, tau, om, eps, LL, LU)
        if on_epoch:
            on_epoch(e, tau, mf, mg)
        if stop:
            stop_epoch = e
            break
    info = dict(omega=om, vd=vd, n_calib=nc, K=K, stopped=stop_epoch >= 0, tau=tau, epochs=epochs,
                stop_epoch=stop_epoch, max_f=mf, max_g=mg, C=Cc, e_scan=e_scan,
                seconds=dict(phases_1_2=t1 - t0, adaptive=time.perf_counter() - t1), threads=threads)
    return counts, cal, LL, LU, info
