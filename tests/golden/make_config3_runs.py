#!/usr/bin/env python
"""Writes the expected end state of the whole method on the two large
single-query workloads, computed by the CPU oracle alone.

    python tests/golden/make_config3_runs.py [grid4096] [rmat26] [--threads T]

For each graph it runs oracle.kadabra_threads (diameter bound -> omega,
calibration, adaptive epochs of E = 1024 samples each checked on its
snapshot; Section III-A, III-B) with eps = 0.01, delta = 0.1, seed 1, the
balanced delta rule (beta = 1e-3) and the default calibration size, and
stores tau at the stop, the stop epoch, the maxima of f and g at the stop
check, omega, the diameter bound, the balancing constant, and SHA-256
digests of the graph, the calibration counts and the final counters into
tests/golden/<name>_run.json.  Only oracle/ and the input generators are
used: no value here comes from the CUDA library.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1910_11039_gb300 import inputs  # noqa: E402

PARAMS = dict(eps=0.01, delta=0.1, seed=1, epoch_len=1024, delta_rule=1, beta=1e-3)


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8)).hexdigest()


def graph_digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.int64(g.n).tobytes())
    h.update(np.ascontiguousarray(g.offsets, dtype=np.int64).view(np.uint8))
    h.update(np.ascontiguousarray(g.cols, dtype=np.int32).view(np.uint8))
    return h.hexdigest()


def run(name: str, threads: int) -> dict:
    t0 = time.time()
    g = inputs.config_graph(name)
    t_gen = time.time() - t0
    print(f"{name}: n={g.n} nnz={g.nnz} built in {t_gen:.1f} s", flush=True)
    trail = []

    def on_epoch(e, tau, mf, mg):
        trail.append([e, tau, float(mf).hex(), float(mg).hex()])
        print(f"  epoch {e} tau {tau} max_f {mf:.6g} max_g {mg:.6g} ({time.time() - t0:.0f} s)", flush=True)

    counts, cal, LL, LU, info = oracle.kadabra_threads(g, PARAMS["eps"], PARAMS["delta"], seed=PARAMS["seed"],
                                                       epoch_len=PARAMS["epoch_len"],
                                                       delta_rule=PARAMS["delta_rule"], beta=PARAMS["beta"],
                                                       threads=threads, on_epoch=on_epoch)
    out = {
        "graph": name, "n": g.n, "nnz": g.nnz, "graph_sha256": graph_digest(g), "params": PARAMS,
        "omega": float(info["omega"]).hex(), "vertex_diameter": info["vd"], "n_calib": info["n_calib"],
        "sigma_bits": info["K"], "C": float(info["C"]).hex(), "stopped": info["stopped"], "tau": info["tau"],
        "stop_epoch": info["stop_epoch"], "max_f": float(info["max_f"]).hex(), "max_g": float(info["max_g"]).hex(),
        "e_scan": info["e_scan"], "counts_sum": int(counts.sum(dtype=np.uint64)), "counts_sha256": sha(counts),
        "cal_sha256": sha(cal), "epochs": trail, "oracle_seconds": round(time.time() - t0, 1),
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=["grid4096", "rmat26"])
    ap.add_argument("--threads", type=int, default=max(1, len(os.sched_getaffinity(0))))
    a = ap.parse_args()
    for name in a.names:
        res = run(name, a.threads)
        path = os.path.join(HERE, f"{name}_run.json")
        with open(path, "w") as f:
            json.dump(res, f, indent=1)
            f.write("\n")
        print(f"wrote {path}", flush=True)


if __name__ == "__main__":
    main()
