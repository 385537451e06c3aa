"""Pins of the oracle's Grassmann geometry, truncated CG and Newton solve.

The p = 2 stage is pinned by the Ky Fan theorem: over orthonormal n x k
blocks, F_2 = trace(U^T L U) is minimised by the k smallest eigenvectors of
the graph Laplacian, so the solve must reach the sum of the k smallest
eigenvalues (closed forms on the path and the cycle, a dense symmetric
eigensolver on random graphs).  At p < 2 the Newton model is pinned by its
parts: the Riemannian Hessian against central differences of the projected
gradient, truncated CG against the Cauchy decrease it guarantees.  The p < 2
trajectory itself has no closed form ("parity unpinned"); it is checked for
descent and planted-block recovery only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_26975_gb300 import workloads as wl


def dense_graph(Wd):
    n = Wd.shape[0]
    iu, ju = np.nonzero(np.triu(Wd, 1))
    return wl.csr_from_undirected(n, iu, ju, Wd[iu, ju], np.float64)


def laplacian(Wd):
    return np.diag(Wd.sum(axis=1)) - Wd


def test_qf_is_thin_qr_with_positive_diagonal():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 5))
    Q = oracle.qf(A)
    assert np.allclose(Q.T @ Q, np.eye(5), atol=1e-14)
    R = Q.T @ A
    assert np.allclose(np.tril(R, -1), 0, atol=1e-13)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(Q @ R, A, atol=1e-13)
    assert np.allclose(oracle.qf(Q), Q, atol=1e-14)


def test_projection():
    rng = np.random.default_rng(1)
    U = oracle.qf(rng.standard_normal((30, 4)))
    G = rng.standard_normal((30, 4))
    P = oracle.project(U, G)
    assert np.allclose(U.T @ P, 0, atol=1e-13)
    assert np.allclose(oracle.project(U, P), P, atol=1e-13)
    # the removed part lies in span(U)
    assert np.allclose(oracle.qf(np.hstack([U, G - P]))[:, 4:] @ np.zeros((4, 4)), 0)
    assert np.linalg.matrix_rank(np.hstack([U, G - P]), tol=1e-10) == 4


def test_tcg_solves_spd_system_inside_radius():
    rng = np.random.default_rng(2)
    m = 12
    B = rng.standard_normal((m, m))
    A = B @ B.T + m * np.eye(m)
    g = rng.standard_normal((m, 1))
    eta, Heta, its, reason, boundary = oracle.tcg(lambda x: A @ x, g, 1e6, 1.0, 1e-12, 200)
    assert reason == "converged" and not boundary
    assert np.allclose(eta, -np.linalg.solve(A, g), rtol=1e-8, atol=1e-10)
    assert np.allclose(Heta, A @ eta, rtol=1e-8, atol=1e-10)


def test_tcg_radius_and_negative_curvature():
    rng = np.random.default_rng(3)
    m = 10
    B = rng.standard_normal((m, m))
    A = B @ B.T + np.eye(m)
    g = rng.standard_normal((m, 1))
    eta, _, _, reason, boundary = oracle.tcg(lambda x: A @ x, g, 1e-3, 1.0, 0.1, 50)
    assert boundary and reason == "radius"
    assert math.isclose(np.linalg.norm(eta), 1e-3, rel_tol=1e-10)
    # indefinite: first direction -g has negative curvature
    A2 = -np.eye(m)
    eta, Heta, its, reason, boundary = oracle.tcg(lambda x: A2 @ x, g, 0.5, 1.0, 0.1, 50)
    assert reason == "negative_curvature" and its == 1
    assert math.isclose(np.linalg.norm(eta), 0.5, rel_tol=1e-12)
    assert np.allclose(eta, -0.5 * g / np.linalg.norm(g))


def test_riemannian_hessian_is_tangent():
    rng = np.random.default_rng(4)
    n, k = 30, 3
    A = np.triu((rng.random((n, n)) < 0.3) * 1.0, 1)
    g = dense_graph(A + A.T)
    U = oracle.qf(rng.standard_normal((n, k)))
    eta = oracle.project(U, rng.standard_normal((n, k)))
    eg = oracle.euclidean_grad(g, U, 1.5)
    H = oracle.riemannian_hessian(U, eg, oracle.euclidean_hvp(g, U, eta, 1.5), eta)
    assert np.allclose(U.T @ H, 0, atol=1e-12)


@pytest.mark.parametrize("p", [1.3, 1.6, 2.0])
def test_riemannian_hessian_is_derivative_of_projected_gradient(p):
    """For tangent eta, differentiating X -> (I - X X^T) grad F(X) at X = U
    along eta gives (I - U U^T) H eta - (eta U^T + U eta^T) grad F; the
    tangent projection of that is P_U(H eta) - eta (U^T grad F), the
    Riemannian Hessian the solve uses.  Central differences of the Euclidean
    gradient check it (the Weingarten term's sign included) at p < 2, where
    nothing else pins the Newton model."""
    rng = np.random.default_rng(int(p * 10))
    n, k = 25, 3
    A = np.triu((rng.random((n, n)) < 0.3) * rng.uniform(0.5, 1.5, (n, n)), 1)
    g = dense_graph(A + A.T)
    U = oracle.qf(rng.standard_normal((n, k)))
    eta = oracle.project(U, rng.standard_normal((n, k)))

    def field(X):
        return oracle.euclidean_grad(g, X, p) - X @ (X.T @ oracle.euclidean_grad(g, X, p))

    def central(t):
        return (field(U + t * eta) - field(U - t * eta)) / (2 * t)

    # Richardson: |d|^p has a large third derivative where an edge's
    # difference is small, so cancel the central difference's t^2 term
    # (the smallest |u| and edge difference here are ~6e-4)
    t = 1e-6
    fd = oracle.project(U, (4 * central(t / 2) - central(t)) / 3)
    egrad = oracle.euclidean_grad(g, U, p)
    H = oracle.riemannian_hessian(U, egrad, oracle.euclidean_hvp(g, U, eta, p), eta)
    assert np.allclose(H, fd, rtol=1e-7, atol=1e-8 * np.abs(H).max())
    # a flipped curvature term would be far off
    wrong = oracle.project(U, oracle.euclidean_hvp(g, U, eta, p)) + eta @ (U.T @ egrad)
    assert not np.allclose(wrong, fd, rtol=1e-3, atol=1e-4 * np.abs(H).max())


@pytest.mark.parametrize("seed", range(6))
def test_tcg_model_no_worse_than_cauchy_point(seed):
    """Steihaug-Toint truncated CG takes the Cauchy point -tau g (the model's
    minimiser along -g inside the radius) as its first iterate and never
    raises the model afterwards, so it ends at or below the Cauchy point's
    model value, inside the trust region."""
    rng = np.random.default_rng(40 + seed)
    m = 15
    B = rng.standard_normal((m, m))
    A = B @ B.T / m + (rng.uniform(-1.0, 0.5) if seed % 2 else 0.1) * np.eye(m)  # odd seeds: indefinite
    g = rng.standard_normal((m, 1))
    Delta = 10.0 ** rng.uniform(-1.5, 1.0)

    def model(x):
        return (g.T @ x + 0.5 * x.T @ A @ x).item()

    gAg = (g.T @ A @ g).item()
    gn = float(np.linalg.norm(g))
    tau = Delta / gn if gAg <= 0 else min(gn * gn / gAg, Delta / gn)
    m_cauchy = model(-tau * g)
    eta, Heta, its, reason, boundary = oracle.tcg(lambda x: A @ x, g, Delta, 1.0, 0.01, 100)
    assert np.linalg.norm(eta) <= Delta * (1 + 1e-12)
    assert model(eta) <= m_cauchy + 1e-12 * abs(m_cauchy)
    assert np.allclose(Heta, A @ eta, rtol=1e-9, atol=1e-12 * np.abs(Heta).max())


def _solve_p2(g, k, seed=0):
    U0 = wl.orthonormal_block(seed, g.n, k, np.float64)
    opts = oracle.SolveOptions(max_outer=60, gtol_rel=1e-9)
    U, st = oracle.rtr_newton(g, U0, 2.0, opts)
    return U, st


@pytest.mark.parametrize("n,k", [(20, 3), (31, 4)])
def test_p2_path_graph_eigenvalues(n, k):
    Wd = np.zeros((n, n))
    for i in range(n - 1):
        Wd[i, i + 1] = Wd[i + 1, i] = 1.0
    g = dense_graph(Wd)
    U, st = _solve_p2(g, k, seed=n)
    ref = sum(2 - 2 * math.cos(math.pi * j / n) for j in range(k))
    assert math.isclose(oracle.objective(g, U, 2.0), ref, rel_tol=1e-8)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-12)


def test_p2_cycle_graph_eigenvalues():
    n, k = 24, 3
    Wd = np.zeros((n, n))
    for i in range(n):
        Wd[i, (i + 1) % n] = Wd[(i + 1) % n, i] = 1.0
    g = dense_graph(Wd)
    U, st = _solve_p2(g, k, seed=3)
    ref = 0.0 + 2 * (2 - 2 * math.cos(2 * math.pi / n))
    assert math.isclose(oracle.objective(g, U, 2.0), ref, rel_tol=1e-8)


def test_p2_random_graph_matches_dense_eigensolver():
    rng = np.random.default_rng(5)
    n, k = 60, 4
    A = np.triu((rng.random((n, n)) < 0.12) * rng.uniform(0.5, 1.5, (n, n)), 1)
    Wd = A + A.T
    g = dense_graph(Wd)
    U, st = _solve_p2(g, k, seed=9)
    ev = np.linalg.eigvalsh(laplacian(Wd))
    assert math.isclose(oracle.objective(g, U, 2.0), ev[:k].sum(), rel_tol=1e-8)
    assert st["gnorm"] <= 1e-6 * max(1.0, st["gnorm0"])


@pytest.mark.slow
def test_sbm4_continuation_recovers_blocks_and_descends():
    g = wl.make_graph("sbm4", np.float64)
    k = 4
    U0 = wl.orthonormal_block(2000, g.n, k, np.float64)
    U, labels, rc, stages = oracle.solve(g, U0, (2.0, 1.8, 1.6, 1.4, 1.2))
    # planted blocks recovered up to a permutation of the labels
    conf = np.zeros((4, 4), dtype=int)
    np.add.at(conf, (g.labels, labels), 1)
    assert (conf.max(axis=1) >= 240).all()
    assert len(set(conf.argmax(axis=1))) == 4
    # every stage decreases its objective from the warm start
    Uc = U0
    for st in stages:
        assert st["f"] <= oracle.objective(g, Uc, st["p"]) + 1e-12
    # RCut of the p-final clustering is no worse than the p = 2 stage's
    U2, lab2, rc2, _ = oracle.solve(g, U0, (2.0,))
    assert rc <= rc2 * (1 + 1e-9)


def test_alg1_hessian_form_is_exact_on_tangent_vectors_at_p2():
    """Algorithm 1 applies only the sparse-plus-diagonal part of the
    quotient's Hessian.  At p = 2 the dropped rank-two terms of column l are
    combinations of u_l (since <g_D, eta> = 2<u_l, eta_l> = 0 for tangent eta
    and g_D = 2 u_l), so the tangent projection removes them: the Riemannian
    Hessians of the two forms agree, and so do the p = 2 solves (Ky Fan)."""
    rng = np.random.default_rng(12)
    n, k = 40, 3
    A = np.triu((rng.random((n, n)) < 0.2) * rng.uniform(0.5, 1.5, (n, n)), 1)
    Wd = A + A.T
    g = dense_graph(Wd)
    U = wl.orthonormal_block(4, n, k, np.float64)
    eta = oracle.project(U, rng.standard_normal((n, k)))
    egrad = oracle.euclidean_grad(g, U, 2.0)
    h_exact = oracle.riemannian_hessian(U, egrad, oracle.euclidean_hvp(g, U, eta, 2.0), eta)
    h_alg1 = oracle.riemannian_hessian(U, egrad, oracle.alg1_sparse_hvp(g, U, eta, 2.0), eta)
    assert np.allclose(h_alg1, h_exact, rtol=0, atol=1e-12 * np.abs(h_exact).max())
    # for p < 2 the forms differ (the rank-two terms have tangent parts)
    egrad = oracle.euclidean_grad(g, U, 1.5)
    d = oracle.riemannian_hessian(U, egrad, oracle.euclidean_hvp(g, U, eta, 1.5)
                                  - oracle.alg1_sparse_hvp(g, U, eta, 1.5), 0 * eta)
    assert np.linalg.norm(d) > 1e-6 * np.linalg.norm(h_exact)
    opts = oracle.SolveOptions(max_outer=60, gtol_rel=1e-9, hessian="alg1")
    U1, st = oracle.rtr_newton(g, wl.orthonormal_block(9, n, k, np.float64), 2.0, opts)
    ev = np.linalg.eigvalsh(laplacian(Wd))
    assert math.isclose(oracle.objective(g, U1, 2.0), ev[:k].sum(), rel_tol=1e-8)
