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
