"""The seeded input generators: every graph is a valid undirected CSR (both
triangles, sorted rows, no self loops, no duplicates, non-negative weights),
generation is reproducible, and each workload has the shape it is named for."""
import numpy as np
import pytest

from paper_2605_26975_gb300 import workloads as wl


def check_csr(g):
    n = g.n
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.nnz and np.all(np.diff(g.rowptr) >= 0)
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    assert np.all((g.col >= 0) & (g.col < n))
    assert not np.any(rows == g.col)
    for i in range(0, n, max(1, n // 200)):  # sorted, duplicate-free rows (sampled)
        c = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    assert np.all(g.val >= 0)
    # symmetric: the multiset of (i, j, w) equals that of (j, i, w)
    a = np.lexsort((g.col, rows))
    b = np.lexsort((rows, g.col))
    assert np.array_equal(rows[a], g.col[b]) and np.array_equal(g.col[a], rows[b])
    assert np.array_equal(g.val[a], g.val[b])


@pytest.mark.parametrize("r", [10, 12])
def test_delaunay_is_planar_triangulation(r):
    n = 1 << r
    g = wl.delaunay_unit_square(7, n)
    check_csr(g)
    m = g.nnz // 2
    # a planar triangulation of n points in general position has
    # 3n - 3 - h edges, h the points on the convex hull (h >= 3)
    assert 3 * n - 3 - 0.05 * n <= m <= 3 * n - 6
    assert np.all(g.val == 1)
    g2 = wl.delaunay_unit_square(7, n)
    assert np.array_equal(g.col, g2.col)


def test_named_small_workloads():
    g = wl.make_graph("sbm4")
    check_csr(g)
    assert g.n == 1000
    for name in ("delaunay16",):
        assert wl.WORKLOADS[name]["k"] == 4
