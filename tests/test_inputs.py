"""Seeded input generators: CSR well-formedness and determinism."""
import numpy as np
import pytest

from paper_1910_11039_gb300 import inputs as I


def assert_valid_csr(g):
    off, col = g.offsets, g.cols
    assert off.dtype == np.int64 and col.dtype == np.int32
    assert off[0] == 0 and off[-1] == col.size and np.all(np.diff(off) >= 0)
    assert col.size == 0 or (col.min() >= 0 and col.max() < g.n)
    rows = np.repeat(np.arange(g.n), np.diff(off))
    assert not np.any(rows == col), "self-loop"
    # rows strictly ascending -> sorted and duplicate-free
    same_row = rows[1:] == rows[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    # symmetric
    fwd = np.sort(rows.astype(np.int64) * g.n + col)
    bwd = np.sort(col.astype(np.int64) * g.n + rows)
    assert np.array_equal(fwd, bwd)


@pytest.mark.parametrize("name", ["er2000", "rmat12", "rmat14", "grid64", "grid256", "rgg5k"])
def test_config_graphs_are_valid(name):
    g = I.config_graph(name)
    assert_valid_csr(g)


@pytest.mark.parametrize("name", ["er2000", "grid64", "rgg5k"])
def test_lcc_graphs_are_connected(name):
    from scipy.sparse.csgraph import connected_components
    import scipy.sparse as sp
    g = I.config_graph(name)
    a = sp.csr_matrix((np.ones(g.nnz), g.cols, g.offsets), shape=(g.n, g.n))
    assert connected_components(a, directed=False)[0] == 1


def test_generators_are_deterministic():
    a = I.rmat_graph(10, 8, seed=5)
    b = I.rmat_graph(10, 8, seed=5)
    c = I.rmat_graph(10, 8, seed=6)
    assert np.array_equal(a.cols, b.cols) and np.array_equal(a.offsets, b.offsets)
    assert not (a.nnz == c.nnz and np.array_equal(a.cols, c.cols))


def _rmat_native(scale, ef, seed, threads, relabel=True):
    L = I._generator()
    n = 1 << scale
    off = np.empty(n + 1, dtype=np.int64)
    cols = np.empty(2 * ef * n, dtype=np.int32)
    nnz = L.gg_rmat_csr(scale, ef, seed, 0.57, 0.19, 0.19, int(relabel), threads, off.ctypes.data, cols.ctypes.data)
    assert nnz >= 0
    return I.Graph(n, off, cols[:nnz])


def test_rmat_builder_is_independent_of_the_thread_count():
    a = _rmat_native(14, 16, 3, 1)
    b = _rmat_native(14, 16, 3, 5)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)
    assert_valid_csr(a)


def test_rmat_quadrant_frequencies():
    # Without relabelling, an edge lands in the top-left / off-diagonal /
    # bottom-right quadrant of the adjacency matrix with probability a,
    # b + c, d (0.57, 0.38, 0.05).  At one edge draw per vertex duplicates
    # are rare, so the symmetric CSR's entries follow the same split.
    g = _rmat_native(20, 1, 11, 4, relabel=False)
    half = g.n // 2
    rows = np.repeat(np.arange(g.n), g.degrees)
    top_r, top_c = rows >= half, g.cols >= half
    frac = lambda m: float(m.sum()) / g.nnz
    assert abs(frac(~top_r & ~top_c) - 0.57) < 0.01
    assert abs(frac(top_r & top_c) - 0.05) < 0.005
    assert abs(frac(top_r ^ top_c) - 0.38) < 0.01


def test_rmat_relabelling_is_a_permutation_of_the_unrelabelled_graph():
    a = _rmat_native(12, 8, 9, 2, relabel=False)
    b = _rmat_native(12, 8, 9, 2, relabel=True)
    assert a.nnz == b.nnz
    assert np.array_equal(np.sort(a.degrees), np.sort(b.degrees))


def test_small_families():
    for g in [I.path_graph(5), I.star_graph(6), I.cycle_graph(7), I.complete_graph(5),
              I.full_grid_graph(3, 4)]:
        assert_valid_csr(g)
    assert I.cycle_graph(7).nnz == 14 and I.complete_graph(5).nnz == 20
    assert I.full_grid_graph(3, 4).nnz == 2 * (3 * 3 + 2 * 4)


def _rhg_brute(n, k, seed):
    """Adjacency of the random hyperbolic graph by the definition: every pair's
    hyperbolic distance against R (same draws as the generator)."""
    rng = np.random.default_rng(seed)
    alpha, xi = 1.0, 2.0
    R = 2 * np.log(2 * xi * xi * n / (np.pi * k))
    theta = rng.random(n) * 2 * np.pi
    u = rng.random(n)
    r = np.arccosh(1 + u * (np.cosh(alpha * R) - 1)) / alpha
    # hyperbolic law of cosines
    coshd = (np.cosh(r[:, None]) * np.cosh(r[None, :])
             - np.sinh(r[:, None]) * np.sinh(r[None, :]) * np.cos(theta[:, None] - theta[None, :]))
    adj = coshd <= np.cosh(R)
    np.fill_diagonal(adj, False)
    return adj, coshd, np.cosh(R)


@pytest.mark.parametrize("n,k,seed", [(500, 20, 3), (1200, 60, 5)])
def test_rhg_matches_the_definition(n, k, seed):
    g = I.rhg_graph(n, k, seed=seed)
    adj, coshd, coshR = _rhg_brute(n, k, seed)
    got = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(g.offsets))
    got[rows, g.cols] = True
    # pairs within rounding of the threshold may go either way between the
    # two distance formulas; every other pair must agree
    clear = np.abs(coshd - coshR) > 1e-9 * coshR
    assert np.array_equal(got[clear], adj[clear])
    assert (got != adj).sum() <= 2


def test_rhg_degree_law():
    g = I.rhg_graph(1 << 14, 60, seed=1)
    deg = np.diff(g.offsets)
    assert abs(deg.mean() - 60) < 0.15 * 60
    # power law with exponent 3: the largest degree is far above the mean and
    # the share of vertices of degree >= d falls roughly as d^-2
    assert deg.max() > 20 * deg.mean()
    f1 = (deg >= 120).mean()
    f2 = (deg >= 480).mean()
    assert 8 < f1 / max(f2, 1e-9) < 32
