"""The block- and star-wise oracle helpers of the full-size parity tests
(tests/oracle_rows.py) against the whole-graph oracle on small graphs: a
block boundary, a row order or a term the helpers got wrong fails here, on
the CPU, before they are trusted at 8M vertices."""
import numpy as np
import pytest

import oracle
import oracle_rows as orw
from gpu_common import grad_term_scale, hvp_term_scale, star_plus_powerlaw
from paper_2605_26975_gb300 import workloads as wl


def graphs():
    return {
        "grid": wl.grid3d_longrange(2, side=9, frac_long=0.02),
        "hubs": star_plus_powerlaw(3, n=2000),
    }


@pytest.mark.parametrize("name", ["grid", "hubs"])
@pytest.mark.parametrize("p", [2.0, 1.3])
def test_block_and_star_helpers_match_whole_graph_oracle(name, p):
    g = graphs()[name]
    k = 3
    U = wl.orthonormal_block(5, g.n, k).astype(np.float64)
    V = wl.gaussian_block(6, g.n, k).astype(np.float64)
    N, D = orw.oracle_N_D(g, U, p, rows_per_chunk=97)
    N_ref, D_ref = oracle.objective_parts(g, U, p)
    assert np.allclose(N, N_ref, rtol=1e-13, atol=0) and np.array_equal(D, D_ref)
    delta = orw.oracle_delta(g, U, p, rows_per_chunk=97)
    assert np.allclose(delta, oracle.p_laplacian(g, U, p), rtol=1e-13, atol=1e-15)
    gr = orw.oracle_grad(g, U, p, N, D, delta)
    scale = grad_term_scale(oracle, g, U, p)
    assert np.all(np.abs(gr - oracle.euclidean_grad(g, U, p)) <= 1e-13 * scale)
    rows = np.array([0, 1, 7, g.n // 2, g.n - 1, int(np.argmax(np.diff(g.rowptr)))])
    assert np.allclose(orw.oracle_delta_rows(g, U, p, rows), delta[rows], rtol=1e-13, atol=1e-15)
    hv = orw.oracle_hvp_rows(g, U, V, p, rows, N, D, delta)
    hs = hvp_term_scale(oracle, g, U, V, p)[rows]
    assert np.all(np.abs(hv - oracle.euclidean_hvp(g, U, V, p)[rows]) <= 1e-12 * hs)
    assert np.allclose(orw.grad_scale(g, U, p, N, D, rows_per_chunk=97), scale, rtol=1e-12, atol=0)
    assert np.allclose(orw.grad_scale_rows(g, U, p, rows, N, D), scale[rows], rtol=1e-12, atol=0)


def test_star_sparse_part_with_ties():
    # quantised values: ties inside the stars must drop their curvature term
    g = graphs()["hubs"]
    rng = np.random.default_rng(3)
    U = rng.integers(-2, 3, size=(g.n, 2)) * 0.5
    U[:, 0] += 0.1  # keep every column norm positive
    V = rng.standard_normal((g.n, 2))
    p = 1.4
    N, D = oracle.objective_parts(g, U, p)
    delta = oracle.p_laplacian(g, U, p)
    rows = np.arange(0, g.n, 37)
    hv = orw.oracle_hvp_rows(g, U, V, p, rows, N, D, delta)
    hs = hvp_term_scale(oracle, g, U, V, p)[rows]
    assert np.all(np.abs(hv - oracle.euclidean_hvp(g, U, V, p)[rows]) <= 1e-12 * hs)
