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
