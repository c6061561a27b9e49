"""The C-ABI library: it loads, exports every declared symbol, and its host-only
entry points (no device needed) behave as declared."""
import math
import os
import re

import numpy as np
import pytest

from paper_1910_11039_gb300 import build as B
from paper_1910_11039_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def K():
    B.build()
    from paper_1910_11039_gb300 import kadabra
    kadabra.load()
    return kadabra


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(kadabra_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(K):
    lib = K.load()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # the binding declares a signature for each of them
    assert names == set(K.SIGNATURES), names ^ set(K.SIGNATURES)


def test_nm_lists_symbols(K):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", K.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), name


def test_status_strings_and_version(K):
    lib = K.load()
    assert lib.kadabra_abi_version() == 100
    assert lib.kadabra_status_string(0) == b"KADABRA_OK"
    assert lib.kadabra_status_string(4) == b"KADABRA_ERR_SIGMA_OVERFLOW"


def test_params_default(K):
    p = K.params_default()
    assert p.eps == 0.01 and p.delta == 0.1 and p.seed == 1 and p.threads == 1024
    assert p.delta_rule == K.DELTA_BALANCED and p.beta == 1e-3


def test_omega_matches_oracle(K, orc):
    for eps, delta, vd in [(0.05, 0.1, 13), (0.01, 0.1, 17), (0.001, 0.1, 795), (0.02, 0.05, 2), (0.3, 0.5, 1)]:
        assert K.omega(eps, delta, vd) == orc.omega(eps, delta, vd)
    with pytest.raises(K.KadabraError):
        K.omega(0.0, 0.1, 10)
    with pytest.raises(K.KadabraError):
        K.omega(0.1, 1.0, 10)


def test_sigma_bits_matches_oracle(K, orc):
    for n, md in [(2, 1), (2000, 21), (1 << 20, 64854), (4096 * 4096, 4), (10, 0)]:
        assert K.sigma_bits(n, md) == orc.sigma_bits(n, md)


def test_validate_accepts_generated_graphs(K):
    for name in ["er2000", "grid64", "rmat12"]:
        g = I.config_graph(name)
        K.validate_csr(g.n, g.offsets, g.cols)
        K.validate_csr(g.n, g.offsets32(), g.cols)


@pytest.mark.parametrize("case", ["unsorted", "self_loop", "asymmetric", "out_of_range", "bad_offsets",
                                  "duplicate", "n_zero"])
def test_validate_rejects_malformed_csr(K, case):
    g = I.cycle_graph(6)
    off = g.offsets.copy()
    col = g.cols.copy()
    n = g.n
    if case == "unsorted":
        col[0], col[1] = col[1], col[0]
    elif case == "self_loop":
        col[0] = 0
    elif case == "asymmetric":
        # vertex 0's neighbour 1 replaced by 3: 0->3 has no reverse
        col[0] = 3 if col[0] != 3 else 2
        col[0:2] = np.sort(col[0:2])
    elif case == "out_of_range":
        col[-1] = n
    elif case == "bad_offsets":
        off[2] = off[1] - 1
    elif case == "duplicate":
        col[1] = col[0]
    elif case == "n_zero":
        n = 0
    with pytest.raises(K.KadabraError) as ei:
        K.validate_csr(n, off, col)
    assert ei.value.status == 1


def test_graph_load_rejects_before_touching_the_device(K):
    # invalid arguments are refused on the host, so this runs without a GPU
    g = I.cycle_graph(5)
    col = g.cols.copy()
    col[0] = 0
    with pytest.raises(K.KadabraError) as ei:
        K.Graph(g.n, g.offsets, col)
    assert ei.value.status == 1 and "self-loop" in str(ei.value)
    with pytest.raises(K.KadabraError):
        K.Graph(0, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32))


def test_binding_structs_match_the_header_layout(K, tmp_path):
    # Every ctypes structure of the binding has the field offsets and the size
    # that a C compiler gives the header's struct, and the flag constants equal
    # the header's macros: a layout drift would hand the library wrong fields.
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("kadabra_params", K.Params), ("kadabra_query_info", K.QueryInfo),
             ("kadabra_trace_rec", K.TraceRec), ("kadabra_launch_stats", K.LaunchStats)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kadabra.h"', "int main(void) {"]
    want = []
    for cname, cls in pairs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            if fname.startswith("pad"):
                continue
            lines.append(f'printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append(getattr(cls, fname).offset)
    macros = [("KADABRA_GRAPH_DEVICE_PTRS", K.GRAPH_DEVICE_PTRS), ("KADABRA_GRAPH_SKIP_VALIDATE", K.GRAPH_SKIP_VALIDATE),
              ("KADABRA_STRICT_SIGMA", K.STRICT_SIGMA), ("KADABRA_FULL_LOOKAHEAD", K.FULL_LOOKAHEAD),
              ("KADABRA_DELTA_UNIFORM", K.DELTA_UNIFORM), ("KADABRA_DELTA_BALANCED", K.DELTA_BALANCED)]
    for m, v in macros:
        lines.append(f'printf("%zu\\n", (size_t)({m}));')
        want.append(v)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want
