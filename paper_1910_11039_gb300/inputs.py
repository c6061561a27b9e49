"""Seeded synthetic graph generators (inputs only).

Every graph the library is tested or measured on comes from here.  The module
builds undirected, unweighted graphs and returns them as a symmetric CSR with
ascending neighbour lists, no self-loops and no duplicate edges, the input
class the method assumes (Section III: undirected, unweighted graphs;
Section V-A: largest connected component of disconnected inputs).

It holds none of the method's arithmetic: no sampling, no BFS with path
counts, no stopping rule.  Both the CPU oracle and the CUDA library consume
its output, which keeps the two sides independent of each other.

The synthetic families stand in for the paper's workloads (Section V-A):
  * R-MAT with the Graph500 parameters (a, b, c, d) = (0.57, 0.19, 0.19, 0.05),
    which the paper uses for its synthetic experiments and which mimics the
    complex networks of Table I;
  * Erdos-Renyi G(n, p) for the small exact-check case;
  * 2D grids with randomly deleted edges and random geometric graphs as
    high-diameter stand-ins for the road networks of Table I.
"""
from __future__ import annotations

import ctypes
import dataclasses
import functools
import os
import subprocess

import numpy as np

__all__ = [
    "Graph", "csr_from_edges", "largest_component", "er_graph", "rmat_graph",
    "grid_graph", "rgg_graph", "rhg_graph", "path_graph", "star_graph", "cycle_graph",
    "complete_graph", "full_grid_graph", "layered_graph", "config_graph", "CONFIGS",
    "graph_from_spec", "batched_specs", "SERVING_POOL", "serving_requests",
]


@dataclasses.dataclass(frozen=True)
class Graph:
    """Symmetric CSR: ``offsets`` int64[n+1], ``cols`` int32[nnz], rows sorted."""

    n: int
    offsets: np.ndarray
    cols: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def max_degree(self) -> int:
        return int(self.degrees.max()) if self.n else 0

    def offsets32(self) -> np.ndarray:
        if self.nnz >= 2**31:
            raise ValueError("graph too large for int32 offsets")
        return self.offsets.astype(np.int32)


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, name: str = "") -> Graph:
    """Symmetrise an edge list, drop self-loops and duplicates, sort rows."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    keys = np.concatenate([src * n + dst, dst * n + src])
    del src, dst
    keys.sort()
    if keys.size:
        keep = np.empty(keys.size, dtype=bool)
        keep[0] = True
        np.not_equal(keys[1:], keys[:-1], out=keep[1:])
        keys = keys[keep]
    rows = keys // n
    cols = (keys - rows * n).astype(np.int32)
    del keys
    counts = np.bincount(rows, minlength=n)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return Graph(n, offsets, cols, name)


def largest_component(g: Graph) -> Graph:
    """Restrict to the largest connected component (ties: lowest label),
    renumbering vertices in their original relative order."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    if g.n == 0:
        return g
    a = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.cols, g.offsets), shape=(g.n, g.n))
    ncomp, labels = connected_components(a, directed=False)
    if ncomp == 1:
        return g
    sizes = np.bincount(labels)
    keep = labels == int(np.argmax(sizes))
    new_id = np.cumsum(keep) - 1
    deg = np.diff(g.offsets)
    rows = np.repeat(np.arange(g.n), deg)
    emask = keep[rows]
    src = new_id[rows[emask]]
    dst = new_id[g.cols[emask]]
    m = int(keep.sum())
    counts = np.bincount(src, minlength=m)
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    # rows are already grouped and ascending because the renumbering is monotone
    return Graph(m, offsets, dst.astype(np.int32), g.name)


def er_graph(n: int, avg_degree: float, seed: int, lcc: bool = True) -> Graph:
    """Erdos-Renyi G(n, p) with p = avg_degree / (n - 1)."""
    rng = np.random.default_rng(seed)
    p = avg_degree / (n - 1)
    iu, ju = np.triu_indices(n, k=1)
    mask = rng.random(iu.shape[0]) < p
    g = csr_from_edges(n, iu[mask], ju[mask], name=f"er{n}")
    return largest_component(g) if lcc else g


_GEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gen")
_GEN_SRC = os.path.join(_GEN_DIR, "graphgen.c")
_GEN_LIB = os.path.join(_GEN_DIR, "libgraphgen.so")
_gen = None


def build_generator(force: bool = False) -> str:
    """Compile the native R-MAT builder with gcc (in place, next to its source)."""
    if force or not os.path.exists(_GEN_LIB) or os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _GEN_SRC])
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _generator():
    global _gen
    if _gen is None:
        L = ctypes.CDLL(build_generator())
        L.gg_rmat_csr.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.gg_rmat_csr.restype = ctypes.c_int64
        _gen = L
    return _gen


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def rmat_graph(scale: int, edge_factor: int, seed: int,
               abcd=(0.57, 0.19, 0.19, 0.05), relabel: bool = True,
               lcc: bool = False) -> Graph:
    """R-MAT (Chakrabarti et al.) with ``edge_factor * 2**scale`` edge draws,
    no noise, random vertex relabelling, symmetrised and deduplicated, built by
    the native counter-based builder (``gen/graphgen.c``): the graph depends
    only on the arguments, not on the thread count."""
    a, b, c, _ = abcd
    n = 1 << scale
    m = edge_factor * n
    off = np.empty(n + 1, dtype=np.int64)
    cols = np.empty(2 * m, dtype=np.int32)
    nnz = _generator().gg_rmat_csr(scale, edge_factor, seed, a, b, c, int(relabel), _threads(),
                                   off.ctypes.data, cols.ctypes.data)
    if nnz < 0:
        raise MemoryError("R-MAT builder failed")
    g = Graph(n, off, cols[:nnz], name=f"rmat{scale}_ef{edge_factor}")
    return largest_component(g) if lcc else g


def grid_graph(k: int, delete_p: float, seed: int, lcc: bool = True) -> Graph:
    """k x k 4-neighbour grid; each edge deleted independently with prob. delete_p."""
    rng = np.random.default_rng(seed)
    idx = np.arange(k * k, dtype=np.int64).reshape(k, k)
    h_src, h_dst = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    v_src, v_dst = idx[:-1, :].ravel(), idx[1:, :].ravel()
    src = np.concatenate([h_src, v_src])
    dst = np.concatenate([h_dst, v_dst])
    keep = rng.random(src.shape[0]) >= delete_p
    g = csr_from_edges(k * k, src[keep], dst[keep], name=f"grid{k}_del{delete_p}")
    return largest_component(g) if lcc else g


def rgg_graph(n: int, avg_degree: float, seed: int, lcc: bool = False) -> Graph:
    """Random geometric graph in the unit square, radius sqrt(avg_degree/(pi n))."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = float(np.sqrt(avg_degree / (np.pi * n)))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    g = csr_from_edges(n, pairs[:, 0], pairs[:, 1], name=f"rgg{n}")
    return largest_component(g) if lcc else g


def rhg_graph(n: int, avg_degree: float, gamma: float = 3.0, seed: int = 0, lcc: bool = False,
              bands: int = 32) -> Graph:
    """Random hyperbolic graph, threshold model (Krioukov et al. 2010): n
    points in a hyperbolic disk of radius R with uniform angles and radial
    density alpha sinh(alpha r) / (cosh(alpha R) - 1), alpha = (gamma - 1) / 2
    (degree power law with exponent gamma); two points are adjacent when
    their hyperbolic distance is at most R.  R = 2 ln(2 xi^2 n / (pi k)) with
    xi = alpha / (alpha - 1/2) gives expected average degree k (Gugelmann,
    Panagiotou and Peter 2012).
    Neighbours are found band by band (points sorted by angle within radial
    bands of equal size): a point at radius r can only reach a band whose
    lowest radius is b within the angle acos((cosh r cosh b - cosh R) /
    (sinh r sinh b)); it searches only bands whose largest radius is at least
    r (the other endpoint of a pair searches the rest), and every candidate
    pair is confirmed with cosh d = cosh(r1 - r2) + 2 sin^2(dtheta / 2)
    sinh r1 sinh r2."""
    rng = np.random.default_rng(seed)
    alpha = (gamma - 1.0) / 2.0
    xi = alpha / (alpha - 0.5)
    R = 2.0 * np.log(2.0 * xi * xi * n / (np.pi * avg_degree))
    theta = rng.random(n) * (2.0 * np.pi)
    u = rng.random(n)
    r = np.arccosh(1.0 + u * (np.cosh(alpha * R) - 1.0)) / alpha
    cosh_R = np.cosh(R)
    ch, sh = np.cosh(r), np.sinh(r)
    by_r = np.argsort(r, kind="stable")
    srcs, dsts = [], []
    for band in np.array_split(by_r, bands):
        if band.size == 0:
            continue
        b = float(r[band].min())
        top = float(r[band].max())
        order = band[np.argsort(theta[band], kind="stable")]
        th = theta[order]
        ext_th = np.concatenate([th - 2 * np.pi, th, th + 2 * np.pi])
        ext_id = np.concatenate([order, order, order])
        # widest angle at which each point can reach this band
        if b <= 0.0:
            dmax = np.full(n, np.pi)
        else:
            arg = (ch * np.cosh(b) - cosh_R) / (sh * np.sinh(b))
            dmax = np.where(arg <= -1.0, np.pi, np.arccos(np.clip(arg, -1.0, 1.0)))
            dmax = np.where(arg > 1.0, -1.0, dmax)
        # a pair is searched from its endpoint of smaller radius (the other
        # endpoint's band), so only points not above this band search it
        searchers = np.nonzero(r <= top)[0]
        for lo_p in range(0, searchers.size, 1 << 16):
            pts = searchers[lo_p:lo_p + (1 << 16)]
            d = dmax[pts]
            ok = d >= 0.0
            pts, d = pts[ok], d[ok]
            lo = np.searchsorted(ext_th, theta[pts] - d, side="left")
            hi = np.searchsorted(ext_th, theta[pts] + d, side="right")
            cnt = hi - lo
            if cnt.sum() == 0:
                continue
            p_rep = np.repeat(pts, cnt)
            start = np.repeat(lo - np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt)
            q = ext_id[np.arange(cnt.sum()) + start]
            keep = p_rep != q
            p_rep, q = p_rep[keep], q[keep]
            dth = theta[p_rep] - theta[q]
            coshd = np.cosh(r[p_rep] - r[q]) + 2.0 * np.sin(dth / 2.0) ** 2 * sh[p_rep] * sh[q]
            adj = coshd <= cosh_R
            srcs.append(p_rep[adj])
            dsts.append(q[adj])
    src = np.concatenate(srcs) if srcs else np.zeros(0, dtype=np.int64)
    dst = np.concatenate(dsts) if dsts else np.zeros(0, dtype=np.int64)
    g = csr_from_edges(n, src, dst, name=f"rhg{n}")
    return largest_component(g) if lcc else g


def _from_pairs(n, pairs, name):
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return csr_from_edges(n, pairs[:, 0], pairs[:, 1], name=name)


def path_graph(n: int) -> Graph:
    return _from_pairs(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def star_graph(n: int) -> Graph:
    """Centre 0 joined to leaves 1..n-1."""
    return _from_pairs(n, [(0, i) for i in range(1, n)], f"star{n}")


def cycle_graph(n: int) -> Graph:
    return _from_pairs(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def complete_graph(n: int) -> Graph:
    return _from_pairs(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"k{n}")


def full_grid_graph(rows: int, cols: int) -> Graph:
    """Full rows x cols grid, vertex id r*cols + c."""
    pairs = []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                pairs.append((v, v + 1))
            if r + 1 < rows:
                pairs.append((v, v + cols))
    return _from_pairs(rows * cols, pairs, f"fullgrid{rows}x{cols}")


def layered_graph(m: int, k: int, hub_leaves: int = 0) -> Graph:
    """Source 0, then k layers of m vertices with every vertex of a layer
    joined to every vertex of the next, then the sink 1 + k*m joined to the
    whole last layer; there are m**k shortest source-sink paths of length
    k + 1.  With hub_leaves > 0 a separate star (centre 2 + k*m) is added: it
    raises the maximum degree without touching any source-sink path."""
    t = 1 + k * m
    pairs = [(0, 1 + j) for j in range(m)]
    for layer in range(k - 1):
        a = 1 + layer * m
        pairs += [(a + i, a + m + j) for i in range(m) for j in range(m)]
    pairs += [(1 + (k - 1) * m + j, t) for j in range(m)]
    n = t + 1
    if hub_leaves > 0:
        c = n
        pairs += [(c, c + 1 + i) for i in range(hub_leaves)]
        n = c + 1 + hub_leaves
    return _from_pairs(n, pairs, f"layered{m}x{k}")


# Named workloads.  Sizes follow the configurations the library is measured
# on; the "small" entries are the same families at sizes the oracle finishes
# in seconds.
CONFIGS = {
    # G(n=2000, avg degree 8), seed 1, largest component
    "er2000": dict(kind="er", n=2000, avg_degree=8, seed=1, lcc=True),
    # R-MAT scale 20, edge factor 16, Graph500 parameters, generator seed 2
    "rmat20": dict(kind="rmat", scale=20, edge_factor=16, seed=2),
    # 4096 x 4096 grid with 10% of the edges deleted (seed 3), largest component
    "grid4096": dict(kind="grid", k=4096, delete_p=0.1, seed=3, lcc=True),
    # R-MAT scale 26, edge factor 16 (~1.07B edge draws; int64 offsets), generator seed 4
    "rmat26": dict(kind="rmat", scale=26, edge_factor=16, seed=4),
    # small members of the same families
    "rmat12": dict(kind="rmat", scale=12, edge_factor=16, seed=12),
    "rmat14": dict(kind="rmat", scale=14, edge_factor=16, seed=14),
    "rmat16": dict(kind="rmat", scale=16, edge_factor=16, seed=16),
    "grid64": dict(kind="grid", k=64, delete_p=0.1, seed=3, lcc=True),
    "grid256": dict(kind="grid", k=256, delete_p=0.1, seed=3, lcc=True),
    "grid512": dict(kind="grid", k=512, delete_p=0.1, seed=3, lcc=True),
    "rgg5k": dict(kind="rgg", n=5000, avg_degree=10, seed=7, lcc=True),
    # random hyperbolic graphs, power-law exponent 3, |E| = 30 |V| (average degree 60)
    "rhg20": dict(kind="rhg", n=1 << 20, avg_degree=60, gamma=3.0, seed=20),
    "rhg4k": dict(kind="rhg", n=4096, avg_degree=60, gamma=3.0, seed=12),
}


def graph_from_spec(spec: dict, name: str = "") -> Graph:
    """Build a graph from a generator spec ``dict(kind=..., **arguments)``."""
    cfg = dict(spec)
    kind = cfg.pop("kind")
    if kind == "er":
        g = er_graph(**cfg)
    elif kind == "rmat":
        g = rmat_graph(**cfg)
    elif kind == "grid":
        g = grid_graph(**cfg)
    elif kind == "rgg":
        g = rgg_graph(**cfg)
    elif kind == "rhg":
        g = rhg_graph(**cfg)
    else:
        raise KeyError(kind)
    return dataclasses.replace(g, name=name or g.name)


@functools.lru_cache(maxsize=8)
def config_graph(name: str) -> Graph:
    """Build a named workload graph (cached per process)."""
    return graph_from_spec(CONFIGS[name], name)


def batched_specs(count: int = 64, n_rgg: int = 8, seed0: int = 1000,
                  scales=(12, 18), edge_factors=(8, 32), rgg_n=(50_000, 500_000)) -> list[dict]:
    """The many-graphs-of-uneven-size workload: ``count - n_rgg`` R-MAT graphs
    (scale uniform in scales, edge factor uniform in edge_factors, both
    inclusive) followed by ``n_rgg`` random geometric graphs (n uniform in
    rgg_n, average degree 10).  Graph i draws its sizes from a generator
    seeded seed0 + i and its edges with seed seed0 + i.  No largest-component
    restriction: a pair in different components counts as a sample with an
    empty path."""
    specs = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        if i < count - n_rgg:
            specs.append(dict(kind="rmat", scale=int(rng.integers(scales[0], scales[1] + 1)),
                              edge_factor=int(rng.integers(edge_factors[0], edge_factors[1] + 1)), seed=seed0 + i))
        else:
            specs.append(dict(kind="rgg", n=int(rng.integers(rgg_n[0], rgg_n[1] + 1)), avg_degree=10,
                              seed=seed0 + i))
    return specs


# Graphs a query stream draws from: R-MAT scale 14..24 (edge factor 16) and
# perturbed grids 1024^2..4096^2 (10% of the edges deleted, largest component).
SERVING_POOL = {f"rmat{s}": dict(kind="rmat", scale=s, edge_factor=16, seed=100 + s) for s in range(14, 25)}
SERVING_POOL.update({f"grid{k}": dict(kind="grid", k=k, delete_p=0.1, seed=3, lcc=True)
                     for k in (1024, 2048, 3072, 4096)})


def serving_requests(count: int = 2000, rate: float = 20.0, seed: int = 5, pool=None,
                     eps_choices=(0.01, 0.005), delta: float = 0.1) -> list[dict]:
    """A Poisson query stream: exponential inter-arrival gaps with mean
    1/rate seconds, each request's graph uniform over `pool` (names of
    SERVING_POOL) and its eps uniform over eps_choices; request i samples
    with seed `seed` * 1_000_000 + i."""
    pool = list(pool if pool is not None else SERVING_POOL)
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    gi = rng.integers(0, len(pool), count)
    ei = rng.integers(0, len(eps_choices), count)
    return [dict(rid=i, graph=pool[int(gi[i])], eps=float(eps_choices[int(ei[i])]), delta=delta,
                 seed=seed * 1_000_000 + i, arrival=float(arrivals[i])) for i in range(count)]
