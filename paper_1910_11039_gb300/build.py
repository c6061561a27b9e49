"""In-tree build of libkadabra.so for sm_103a (nvcc + g++, no cmake).

The kernels are compiled for ``sm_103a`` only; the host side of the C ABI is
compiled with ``-ffp-contract=off`` so that its double arithmetic (omega,
delta calibration) is the plain IEEE sequence written in the source.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "kadabra")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libkadabra.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wno-unused-function",
             "-I", INCLUDE, "-I", CSRC]

# (source, compiler, extra flags)
UNITS = [
    ("sample_kernel.cu", "nvcc", []),
    ("check_kernel.cu", "nvcc", ["-fmad=false"]),
    ("sample_static.cu", "nvcc", []),
    ("graph_kernels.cu", "nvcc", []),
    ("kadabra_api.cpp", "cxx", []),
]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(os.path.realpath(nv)))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "kadabra.h"), "rb") as f:
        h.update(f.read())
    h.update(repr((ARCH, NVCC_FLAGS, CXX_FLAGS, UNITS)).encode())
    return h.hexdigest()


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile libkadabra.so if its sources changed; return its path."""
    stamp = os.path.join(LIBDIR, ".stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    cxx = os.environ.get("CXX", "g++")
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    jobs = []
    objs = []
    for src, comp, extra in UNITS:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        path = os.path.join(CSRC, src)
        if comp == "nvcc":
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", path, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
        else:
            cmd = [cxx, *CXX_FLAGS, *extra, "-I", os.path.join(home, "include"), "-c", path, "-o", obj]
        jobs.append(cmd)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), jobs))
    if ptxas_info:
        for o in outs:
            if o.strip():
                print(o, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    _run([nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-ldl"], verbose)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
