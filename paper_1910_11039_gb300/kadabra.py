"""Python binding of libkadabra.so (argument marshalling only).

Every function here forwards to the C entry point of the same name in
``include/kadabra.h``; all sampling, stop checks and result computation run
in the library's CUDA kernels.  There is no Python or CPU fallback: if the
shared library is missing the first call raises.

Streams: ``stream=None`` means torch's current CUDA stream when torch sees a
device, else the legacy default stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libkadabra.so")

OK = 0
STATUS = {0: "KADABRA_OK", 1: "KADABRA_ERR_INVALID_ARG", 2: "KADABRA_ERR_OOM", 3: "KADABRA_ERR_CUDA",
          4: "KADABRA_ERR_SIGMA_OVERFLOW", 5: "KADABRA_ERR_COUNTER_OVERFLOW", 6: "KADABRA_ERR_TIMEOUT",
          7: "KADABRA_ERR_STATE", 8: "KADABRA_ERR_NO_DEVICE", 9: "KADABRA_ERR_DEPTH"}

GRAPH_DEVICE_PTRS = 1
GRAPH_SKIP_VALIDATE = 2
STRICT_SIGMA = 1
FULL_LOOKAHEAD = 2
DELTA_UNIFORM = 0
DELTA_BALANCED = 1


class KadabraError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("delta", C.c_double), ("seed", C.c_uint64),
                ("vertex_diameter", C.c_int64), ("n_calib", C.c_int64), ("delta_rule", C.c_int32),
                ("flags", C.c_uint32), ("beta", C.c_double), ("slots", C.c_int32),
                ("threads", C.c_int32), ("scratch_fraction", C.c_double), ("queue_cap", C.c_int64),
                ("coop_edges", C.c_int64), ("probe_edges", C.c_int64)]


class QueryInfo(C.Structure):
    _fields_ = [("omega", C.c_double), ("omega_ceil", C.c_uint64), ("vertex_diameter", C.c_int64),
                ("n_calib", C.c_int64), ("sigma_bits", C.c_int32), ("stopped", C.c_int32),
                ("tau", C.c_uint64), ("epochs", C.c_int64), ("stop_epoch", C.c_int64),
                ("max_f", C.c_double), ("max_g", C.c_double), ("balance_C", C.c_double),
                ("samples", C.c_uint64), ("connected", C.c_uint64), ("e_scan", C.c_uint64),
                ("expanded", C.c_uint64), ("touched", C.c_uint64), ("interior", C.c_uint64),
                ("walk_scan", C.c_uint64), ("scaled", C.c_uint64), ("device_error", C.c_uint32),
                ("slots", C.c_int32), ("threads", C.c_int32), ("offsets_64", C.c_int32),
                ("budget_classes", C.c_int32), ("stop_ns", C.c_uint64), ("phase", C.c_int32),
                ("pad0", C.c_int32), ("cal_done", C.c_uint64), ("device_bytes", C.c_uint64),
                ("launches", C.c_int64), ("diameter_ms", C.c_double), ("calibration_ms", C.c_double),
                ("queue_cap", C.c_int64), ("spill_slots", C.c_int32), ("vd_exact", C.c_int32),
                ("vd_searches", C.c_int64)]


class TraceRec(C.Structure):
    _fields_ = [("s", C.c_int64), ("t", C.c_int64), ("d", C.c_int64), ("sigma_lo", C.c_uint64),
                ("sigma_hi", C.c_uint64), ("meet_size", C.c_int64), ("chosen", C.c_int64),
                ("e_scan", C.c_int64), ("n_interior", C.c_int64), ("scaled", C.c_int32),
                ("overflow", C.c_int32), ("ns", C.c_int64), ("phase_ns", C.c_int64 * 4)]

    @property
    def sigma(self) -> int:
        return (int(self.sigma_hi) << 64) | int(self.sigma_lo)


class LaunchStats(C.Structure):
    _fields_ = [("ms", C.c_float), ("samples", C.c_uint64), ("connected", C.c_uint64),
                ("e_scan", C.c_uint64), ("expanded", C.c_uint64), ("touched", C.c_uint64),
                ("interior", C.c_uint64), ("walk_scan", C.c_uint64), ("grid", C.c_int32),
                ("threads", C.c_int32)]


_P = C.c_void_p
_I64 = C.c_int64
_U64 = C.c_uint64
_ST = C.c_int

# name -> (restype, argtypes); every name declared in include/kadabra.h
SIGNATURES = {
    "kadabra_last_error": (C.c_char_p, []),
    "kadabra_status_string": (C.c_char_p, [_ST]),
    "kadabra_abi_version": (C.c_int, []),
    "kadabra_params_default": (None, [C.POINTER(Params)]),
    "kadabra_validate_csr": (_ST, [_I64, _I64, _P, C.c_int, _P]),
    "kadabra_omega": (_ST, [C.c_double, C.c_double, _I64, C.POINTER(C.c_double)]),
    "kadabra_sigma_bits": (C.c_int, [_I64, _I64]),
    "kadabra_graph_load": (_ST, [_I64, _I64, _P, C.c_int, _P, C.c_uint32, _P, C.POINTER(_P)]),
    "kadabra_graph_free": (_ST, [_P]),
    "kadabra_graph_info": (_ST, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(C.c_int)]),
    "kadabra_calibrate": (_ST, [_P, C.POINTER(Params), _P, C.POINTER(_P)]),
    "kadabra_query_free": (_ST, [_P]),
    "kadabra_sample_epoch": (_ST, [_P, _I64, _P]),
    "kadabra_check_stop": (_ST, [_P, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double), _P]),
    "kadabra_check_stop_async": (_ST, [_P, _P]),
    "kadabra_run": (_ST, [_P, _I64, _I64, _I64, _P, C.POINTER(C.c_int)]),
    "kadabra_run_pipelined": (_ST, [_P, _I64, C.c_int, _P]),
    "kadabra_query_reset": (_ST, [_P, _P]),
    "kadabra_result": (_ST, [_P, _P, _P, C.POINTER(_U64), C.POINTER(_I64), _P]),
    "kadabra_query_get_info": (_ST, [_P, C.POINTER(QueryInfo), _P]),
    "kadabra_query_budgets": (_ST, [_P, _P, _P, _P, _P]),
    "kadabra_sample_trace": (_ST, [_P, C.c_int, _U64, _I64, _P, _P, _I64, _P]),
    "kadabra_last_launch": (_ST, [_P, C.POINTER(LaunchStats)]),
    "kadabra_launch_log": (_ST, [_P, _I64, _P, C.POINTER(_I64)]),
    "kadabra_sample_static": (_ST, [_P, _U64, C.c_int, _U64, _I64, _P, _P]),
    "kadabra_sample_range": (_ST, [_P, C.c_int, _U64, _I64, _P, _P]),
    "kadabra_absorb": (_ST, [_P, _P, _U64, _P]),
    "kadabra_sample_range_log": (_ST, [_P, C.c_int, _U64, _I64, _P, C.c_uint32, _P, _P]),
    "kadabra_absorb_log": (_ST, [_P, _P, _U64, _U64, _P]),
    "kadabra_pipeline_begin": (_ST, [_P, _I64, C.c_int, _P]),
    "kadabra_run_graph": (_ST, [_P, _I64, C.c_int, _I64, _P, C.POINTER(C.c_int)]),
    "kadabra_batch_set_policy": (_ST, [_P, C.c_int]),
    "kadabra_batch_poll": (_ST, [_P, _P, _I64, _P]),
    "kadabra_batch_set_spin_limit": (_ST, [_P, _U64]),
    "kadabra_batch_info": (_ST, [_P, _P, _P, _P]),
    "kadabra_query_restore": (_ST, [_P, _P, _U64, _I64, _P]),
    "kadabra_query_create": (_ST, [_P, _P, _P, _P]),
    "kadabra_calibration_begin": (_ST, [_P, _P]),
    "kadabra_calibration_finish": (_ST, [_P, _P]),
    "kadabra_device_clock": (_ST, [C.POINTER(_U64), _P]),
    "kadabra_batch_create": (_ST, [_I64, C.c_int32, C.c_int32, C.c_int, C.POINTER(_P)]),
    "kadabra_batch_free": (_ST, [_P]),
    "kadabra_batch_step": (_ST, [_P, _P, _I64, _U64, _P]),
    "kadabra_batch_last_ms": (_ST, [_P, C.POINTER(C.c_float)]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libkadabra.so (built by ``paper_1910_11039_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libkadabra.so not built ({p}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st):
    if st != OK:
        raise KadabraError(st, load().kadabra_last_error().decode())


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if hasattr(s, "cuda_stream"):
        return C.c_void_p(s.cuda_stream)
    return C.c_void_p(int(s))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(int(a))


# ---- host utilities ----------------------------------------------------------

def params_default(**kw) -> Params:
    p = Params()
    load().kadabra_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def validate_csr(n, offsets, cols):
    off = np.ascontiguousarray(offsets)
    col = np.ascontiguousarray(cols, dtype=np.int32)
    _check(load().kadabra_validate_csr(n, int(off[-1]) if off.size else 0, _ptr(off),
                                       1 if off.dtype == np.int64 else 0, _ptr(col)))


def omega(eps, delta, vertex_diameter) -> float:
    out = C.c_double()
    _check(load().kadabra_omega(eps, delta, vertex_diameter, C.byref(out)))
    return out.value


def device_clock(stream=None) -> int:
    """Device global timer in ns (the clock of QueryInfo.stop_ns)."""
    v = _U64()
    _check(load().kadabra_device_clock(C.byref(v), _stream(stream)))
    return v.value


def sigma_bits(n, max_degree) -> int:
    return load().kadabra_sigma_bits(n, max_degree)


# ---- graph and query handles ------------------------------------------------

class Graph:
    """Library-owned device copy of a CSR graph (kadabra_graph_load)."""

    def __init__(self, n, offsets, cols, offsets_64=None, device_ptrs=False, skip_validate=False, stream=None,
                 nnz=None):
        lib = load()
        self.handle = C.c_void_p()
        flags = (GRAPH_DEVICE_PTRS if device_ptrs else 0) | (GRAPH_SKIP_VALIDATE if skip_validate else 0)
        if device_ptrs:
            # torch tensors (or raw pointers with explicit nnz / offsets_64)
            off_p = offsets.data_ptr() if hasattr(offsets, "data_ptr") else int(offsets)
            col_p = cols.data_ptr() if hasattr(cols, "data_ptr") else int(cols)
            if offsets_64 is None:
                offsets_64 = str(getattr(offsets, "dtype", "")).endswith("int64")
            if nnz is None:
                nnz = int(offsets[-1])
            self._keep = (offsets, cols)
            _check(lib.kadabra_graph_load(n, nnz, C.c_void_p(off_p), int(bool(offsets_64)), C.c_void_p(col_p),
                                          flags, _stream(stream), C.byref(self.handle)))
        else:
            if offsets_64 is None:
                offsets_64 = offsets.dtype == np.int64
            off = np.ascontiguousarray(offsets, dtype=np.int64 if offsets_64 else np.int32)
            col = np.ascontiguousarray(cols, dtype=np.int32)
            nnz = int(off[-1])
            _check(lib.kadabra_graph_load(n, nnz, _ptr(off), int(bool(offsets_64)), _ptr(col), flags,
                                          _stream(stream), C.byref(self.handle)))
        self.n = n

    @classmethod
    def from_inputs(cls, g, offsets_64=False, **kw):
        off = g.offsets if offsets_64 else g.offsets32()
        return cls(g.n, off, g.cols, offsets_64=offsets_64, **kw)

    def info(self):
        n, nnz, md, o64 = _I64(), _I64(), _I64(), C.c_int()
        _check(load().kadabra_graph_info(self.handle, C.byref(n), C.byref(nnz), C.byref(md), C.byref(o64)))
        return dict(n=n.value, nnz=nnz.value, max_degree=md.value, offsets_64=o64.value)

    def free(self):
        if self.handle:
            load().kadabra_graph_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Query:
    """One betweenness query: kadabra_calibrate and the calls on its result."""

    def __init__(self, graph: Graph, params: Params | None = None, stream=None, calibrate=True, **kw):
        """calibrate=True: kadabra_calibrate (phases 1 and 2 now);
        calibrate=False: kadabra_query_create (phase 1 only; calibrate in a
        batch with calibration_begin / Batch.step / calibration_finish)."""
        self.graph = graph
        p = params if params is not None else params_default()
        for k, v in kw.items():
            setattr(p, k, v)
        self.params = p
        self.handle = C.c_void_p()
        fn = load().kadabra_calibrate if calibrate else load().kadabra_query_create
        _check(fn(graph.handle, C.byref(p), _stream(stream), C.byref(self.handle)))

    def checkpoint(self, stream=None) -> dict:
        """The query's adaptive state (counters, tau, epochs checked) and the
        parameters a restored query must share."""
        res = self.result(btilde=False, stream=stream)
        inf = self.info(stream)
        p = self.params
        return {"counts": res["counts"].astype(np.uint32), "tau": int(res["tau"]), "epochs": int(inf.epochs),
                "eps": p.eps, "delta": p.delta, "seed": int(p.seed), "n_calib": int(inf.n_calib),
                "delta_rule": int(p.delta_rule), "vertex_diameter": int(inf.vertex_diameter)}

    def restore(self, ckpt: dict, stream=None):
        """Continue from a checkpoint taken on a query with the same parameters."""
        inf = self.info(stream)
        p = self.params
        if (ckpt["eps"], ckpt["delta"], ckpt["seed"], ckpt["delta_rule"]) != (p.eps, p.delta, int(p.seed),
                                                                              int(p.delta_rule)) \
                or ckpt["n_calib"] != inf.n_calib or ckpt["vertex_diameter"] != inf.vertex_diameter:
            raise ValueError("checkpoint taken with other query parameters")
        counts = np.ascontiguousarray(ckpt["counts"], dtype=np.uint32)
        if counts.shape != (self.graph.n,):
            raise ValueError("checkpoint counters do not match the graph")
        _check(load().kadabra_query_restore(self.handle, _ptr(counts), int(ckpt["tau"]), int(ckpt["epochs"]),
                                            _stream(stream)))

    def calibration_begin(self, stream=None):
        _check(load().kadabra_calibration_begin(self.handle, _stream(stream)))

    def calibration_finish(self, stream=None):
        _check(load().kadabra_calibration_finish(self.handle, _stream(stream)))

    def sample_epoch(self, n_samples, stream=None):
        _check(load().kadabra_sample_epoch(self.handle, n_samples, _stream(stream)))

    def check_stop(self, stream=None):
        st, mf, mg = C.c_int(), C.c_double(), C.c_double()
        _check(load().kadabra_check_stop(self.handle, C.byref(st), C.byref(mf), C.byref(mg), _stream(stream)))
        return bool(st.value), mf.value, mg.value

    def check_stop_async(self, stream=None):
        _check(load().kadabra_check_stop_async(self.handle, _stream(stream)))

    def run(self, epoch_len, max_epochs=1 << 30, sync_every=4, stream=None) -> bool:
        st = C.c_int()
        _check(load().kadabra_run(self.handle, epoch_len, max_epochs, sync_every, _stream(stream), C.byref(st)))
        return bool(st.value)

    def run_pipelined(self, epoch_len, frames=8, stream=None):
        """Whole adaptive phase as one persistent launch (async)."""
        _check(load().kadabra_run_pipelined(self.handle, epoch_len, frames, _stream(stream)))

    def sample_range(self, tag, first, count, counts_device_ptr, stream=None):
        """Add the interior vertices of samples [first, first+count) to a
        caller-owned device counter array (the query's own state is untouched)."""
        _check(load().kadabra_sample_range(self.handle, tag, first, count, C.c_void_p(int(counts_device_ptr)),
                                           _stream(stream)))

    def absorb(self, delta_device_ptr, samples, stream=None):
        """c~ += delta, tau += samples (the epoch aggregate of a sharded run)."""
        _check(load().kadabra_absorb(self.handle, C.c_void_p(int(delta_device_ptr)), samples, _stream(stream)))

    def sample_range_log(self, tag, first, count, log_device_ptr, log_cap, len_device_ptr, stream=None):
        """Append the interior vertices of samples [first, first+count) to a
        caller-owned device log; the device word at len_device_ptr receives
        the number appended (above log_cap: the log overflowed)."""
        _check(load().kadabra_sample_range_log(self.handle, tag, first, count, C.c_void_p(int(log_device_ptr)),
                                               log_cap, C.c_void_p(int(len_device_ptr)), _stream(stream)))

    def absorb_log(self, log_device_ptr, length, samples, stream=None):
        """c~[x] += 1 for every entry x of a device log, tau += samples."""
        _check(load().kadabra_absorb_log(self.handle, C.c_void_p(int(log_device_ptr)), length, samples,
                                         _stream(stream)))

    def run_graph(self, epoch_len, epochs_per_graph=4, max_epochs=1 << 30, stream=None) -> bool:
        """Stream-ordered epochs replayed from a captured CUDA graph."""
        st = C.c_int()
        _check(load().kadabra_run_graph(self.handle, epoch_len, epochs_per_graph, max_epochs, _stream(stream),
                                        C.byref(st)))
        return bool(st.value)

    def pipeline_begin(self, epoch_len, frames=8, stream=None):
        _check(load().kadabra_pipeline_begin(self.handle, epoch_len, frames, _stream(stream)))

    def reset(self, stream=None):
        _check(load().kadabra_query_reset(self.handle, _stream(stream)))

    def result(self, btilde=True, counts=True, stream=None):
        n = self.graph.n
        b = np.zeros(n, dtype=np.float64) if btilde else None
        c = np.zeros(n, dtype=np.uint32) if counts else None
        tau, se = _U64(), _I64()
        _check(load().kadabra_result(self.handle, _ptr(b), _ptr(c), C.byref(tau), C.byref(se), _stream(stream)))
        return dict(btilde=b, counts=c, tau=tau.value, stop_epoch=se.value)

    def result_into(self, btilde_ptr, counts_ptr, stream=None):
        """Write the result to caller-owned host memory (pinned buffers)."""
        tau, se = _U64(), _I64()
        _check(load().kadabra_result(self.handle, _ptr(btilde_ptr), _ptr(counts_ptr), C.byref(tau), C.byref(se),
                                     _stream(stream)))
        return tau.value, se.value

    def info(self, stream=None) -> QueryInfo:
        I = QueryInfo()
        _check(load().kadabra_query_get_info(self.handle, C.byref(I), _stream(stream)))
        return I

    def budgets(self, stream=None):
        n = self.graph.n
        LL = np.zeros(n, dtype=np.float64)
        LU = np.zeros(n, dtype=np.float64)
        cal = np.zeros(n, dtype=np.uint32)
        _check(load().kadabra_query_budgets(self.handle, _ptr(LL), _ptr(LU), _ptr(cal), _stream(stream)))
        return LL, LU, cal

    def sample_trace(self, tag, first, count, path_cap=0, stream=None):
        recs = (TraceRec * count)()
        paths = np.zeros((count, path_cap), dtype=np.int32) if path_cap > 0 else None
        _check(load().kadabra_sample_trace(self.handle, tag, first, count, C.cast(recs, C.c_void_p), _ptr(paths),
                                           path_cap, _stream(stream)))
        return list(recs), paths

    def last_launch(self) -> LaunchStats:
        s = LaunchStats()
        _check(load().kadabra_last_launch(self.handle, C.byref(s)))
        return s

    def launch_log(self, max_entries=256):
        arr = (LaunchStats * max_entries)()
        got = _I64()
        _check(load().kadabra_launch_log(self.handle, max_entries, C.cast(arr, C.c_void_p), C.byref(got)))
        return list(arr[:got.value])

    def free(self):
        if self.handle:
            load().kadabra_query_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sample_static(graph: Graph, seed, tag, first, count, counts_device_ptr, stream=None):
    """kadabra_sample_static: sampling with the library's fixed scratch array
    (no device allocation); adds interior-vertex counts to a caller-owned
    device array."""
    _check(load().kadabra_sample_static(graph.handle, seed, tag, first, count, C.c_void_p(int(counts_device_ptr)),
                                        _stream(stream)))


class Batch:
    """Sampling scratch shared by many queries stepped in one launch."""

    ROUND_ROBIN, IN_ORDER = 0, 1

    def __init__(self, max_n, slots=0, threads=1024, offsets_64=False, policy=0):
        self.handle = C.c_void_p()
        _check(load().kadabra_batch_create(max_n, slots, threads, int(bool(offsets_64)), C.byref(self.handle)))
        self.max_n = max_n
        self.threads = threads
        if policy:
            self.set_policy(policy)

    def info(self) -> dict:
        sl, th, mn = C.c_int32(), C.c_int32(), _I64()
        _check(load().kadabra_batch_info(self.handle, C.byref(sl), C.byref(th), C.byref(mn)))
        return dict(slots=sl.value, threads=th.value, max_n=mn.value)

    def set_spin_limit(self, polls):
        _check(load().kadabra_batch_set_spin_limit(self.handle, int(polls)))

    def set_policy(self, policy):
        _check(load().kadabra_batch_set_policy(self.handle, int(policy)))
        self.policy = policy

    def step(self, queries, sample_budget=0, stream=None):
        arr = (C.c_void_p * len(queries))(*[q.handle.value for q in queries])
        _check(load().kadabra_batch_step(self.handle, C.cast(arr, C.c_void_p), len(queries), sample_budget,
                                         _stream(stream)))

    def poll(self, count, stream=None) -> np.ndarray:
        """States of the last step's queries: 0 running, 1 calibration
        complete, 2 stopped."""
        out = np.zeros(count, dtype=np.int32)
        _check(load().kadabra_batch_poll(self.handle, _ptr(out), count, _stream(stream)))
        return out

    def last_ms(self) -> float:
        ms = C.c_float()
        _check(load().kadabra_batch_last_ms(self.handle, C.byref(ms)))
        return ms.value

    def free(self):
        if self.handle:
            load().kadabra_batch_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def save_checkpoint(path, ckpt: dict):
    """Write a checkpoint (Query.checkpoint()) to an .npz file."""
    np.savez(path, **{k: np.asarray(v) for k, v in ckpt.items()})


def load_checkpoint(path) -> dict:
    with np.load(path) as z:
        out = {k: z[k] for k in z.files}
    for k in ("tau", "epochs", "seed", "n_calib", "delta_rule", "vertex_diameter"):
        out[k] = int(out[k])
    for k in ("eps", "delta"):
        out[k] = float(out[k])
    return out


# C-ABI names, for callers that prefer the flat interface
def graph_load(n, offsets, cols, **kw) -> Graph:
    return Graph(n, offsets, cols, **kw)


def calibrate(graph: Graph, params: Params | None = None, stream=None, **kw) -> Query:
    return Query(graph, params, stream, **kw)


def sample_epoch(q: Query, n_samples, stream=None):
    q.sample_epoch(n_samples, stream)


def check_stop(q: Query, stream=None):
    return q.check_stop(stream)


def result(q: Query, stream=None):
    return q.result(stream=stream)
