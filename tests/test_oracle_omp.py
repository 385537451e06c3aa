"""Pins of the all-core FP64 C oracle (oracle/plap_omp.c): closed forms on a
two-vertex graph and a two-level vector, and agreement with the numpy oracle
(itself pinned by tests/test_oracle_plap.py) on ragged graphs with hubs, ties
and zero entries, at p = 2 and below."""
import numpy as np
import pytest

import oracle
from gpu_common import star_plus_powerlaw, with_isolated
from oracle import omp
from paper_2605_26975_gb300 import workloads as wl


@pytest.fixture(scope="module", autouse=True)
def built():
    omp.build()
    assert omp.threads() >= 1


@pytest.mark.parametrize("p", [2.0, 1.5, 1.1])
def test_two_vertex_closed_form(p):
    w = 0.7
    g = wl.csr_from_undirected(2, np.array([0]), np.array([1]), np.array([w]), np.float64)
    F, N, D, grad = omp.evaluate(g, np.array([[1.0], [-1.0]]), p)
    assert abs(F - 2.0 ** (p - 1.0) * w) <= 1e-15 * F          # w 2^p / (1 + 1)
    assert abs(N[0] - w * 2.0 ** p) <= 1e-15 * N[0] and D[0] == 2.0
    # u = (a, b): dF/da = p w phi_p(a-b)/D - p w |a-b|^p phi_p(a)/D^2
    a, b = 0.8, -0.3
    F, N, D, grad = omp.evaluate(g, np.array([[a], [b]]), p)
    Dab = abs(a) ** p + abs(b) ** p
    ph = lambda x: np.sign(x) * abs(x) ** (p - 1)
    ga = p * w * ph(a - b) / Dab - p * w * abs(a - b) ** p * ph(a) / Dab ** 2
    gb = p * w * ph(b - a) / Dab - p * w * abs(a - b) ** p * ph(b) / Dab ** 2
    assert np.allclose(grad[:, 0], [ga, gb], rtol=1e-14, atol=0)


@pytest.mark.parametrize("p", [2.0, 1.3])
def test_two_level_vector(p):
    # u = a on A, b elsewhere: N = cut(A) |a - b|^p, D = |A||a|^p + |A'||b|^p
    g = wl.sbm_sampled(np.random.default_rng(3), 300, 3, 8.0, 0.8).astype(np.float64)
    A = np.arange(g.n) < 120
    a, b = 0.9, -0.4
    u = np.where(A, a, b)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    cut = g.val[A[rows] & ~A[g.col]].sum()
    F, N, D, _ = omp.evaluate(g, u, p, grad=False)
    assert abs(N[0] - cut * abs(a - b) ** p) <= 1e-12 * N[0]
    assert abs(D[0] - (A.sum() * abs(a) ** p + (~A).sum() * abs(b) ** p)) <= 1e-13 * D[0]


def graphs():
    return {"sbm": wl.sbm_sampled(np.random.default_rng(1), 800, 4, 10.0, 0.85),
            "hubs": star_plus_powerlaw(3, n=3000), "isolated": with_isolated(4, n=900)}


@pytest.mark.parametrize("name", ["sbm", "hubs", "isolated"])
@pytest.mark.parametrize("p", [2.0, 1.6, 1.1])
@pytest.mark.parametrize("ties", [False, True])
def test_matches_numpy_oracle(name, p, ties):
    g = graphs()[name]
    k = 5
    rng = np.random.default_rng(7)
    U = (rng.integers(-3, 4, size=(g.n, k)) * 0.25 + 0.01 * (np.arange(k) == 0) if ties
         else wl.orthonormal_block(8, g.n, k).astype(np.float64))
    V = rng.standard_normal((g.n, k))
    F, N, D, grad = omp.evaluate(g, U, p)
    N_ref, D_ref = oracle.objective_parts(g, U, p)
    assert np.allclose(N, N_ref, rtol=1e-12, atol=0) and np.allclose(D, D_ref, rtol=1e-13, atol=0)
    assert abs(F - oracle.objective(g, U, p)) <= 1e-12 * F
    g_ref = oracle.euclidean_grad(g, U, p)
    assert np.linalg.norm(grad - g_ref) <= 1e-12 * np.linalg.norm(g_ref)
    h_ref = oracle.euclidean_hvp(g, U, V, p)
    assert np.linalg.norm(omp.hvp(g, U, V, p) - h_ref) <= 1e-12 * np.linalg.norm(h_ref)
