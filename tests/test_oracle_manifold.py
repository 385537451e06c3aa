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


# ---- p < 2 stages pinned on graphs with k connected components: F_p >= 0,
# and F_p = 0 exactly when every column is constant on every component, so
# the span of the component indicators is the global minimum for every p.
# (F_p is not smooth at ties for p < 2, so the approach is slow: the pins are
# bounds, with margins over what the reading reaches.)
def components_graph(sizes, seed):
    """Cycles with random chords, one per size, weights U[0.5, 1.5]: exactly
    len(sizes) connected components.  Returns the graph and each vertex's
    component."""
    rng = np.random.default_rng(seed)
    rows, cols, off = [], [], 0
    for m in sizes:
        a = np.arange(m)
        rows += list(off + a)
        cols += list(off + (a + 1) % m)
        ch = rng.integers(0, m, (m, 2))
        ch = ch[ch[:, 0] != ch[:, 1]]
        rows += list(off + ch[:, 0])
        cols += list(off + ch[:, 1])
        off += m
    r, c = np.array(rows), np.array(cols)
    e = np.unique(np.stack([np.minimum(r, c), np.maximum(r, c)], 1), axis=0)
    g = wl.csr_from_undirected(off, e[:, 0], e[:, 1], rng.uniform(0.5, 1.5, len(e)), np.float64)
    return g, np.repeat(np.arange(len(sizes)), sizes)


def sin_largest_angle(U, V):
    """sin of the largest principal angle between span(U) and span(V)."""
    Qu, Qv = oracle.qf(U), oracle.qf(V)
    return np.linalg.norm(Qu - Qv @ (Qv.T @ Qu), 2)


@pytest.mark.parametrize("p,f_ratio,angle", [(1.5, 1e-3, 0.02), (1.2, 0.05, 0.15)])
def test_p_below_2_stage_approaches_the_component_span(p, f_ratio, angle):
    g, comp = components_graph([30, 24, 36], 3)
    k = 3
    ind = np.zeros((g.n, k))
    ind[np.arange(g.n), comp] = 1.0
    U0 = oracle.qf(ind + 0.2 * np.random.default_rng(5).standard_normal(ind.shape))
    assert sin_largest_angle(U0, ind) > 0.3
    U, st = oracle.rtr_newton(g, U0, p, oracle.SolveOptions(max_outer=100, gtol_rel=1e-9))
    F0, F = oracle.objective(g, U0, p), oracle.objective(g, U, p)
    assert 0.0 <= F <= f_ratio * F0, (F, F0)
    assert sin_largest_angle(U, ind) <= angle
    labels = oracle.kmeans(U, k)[0]
    assert len(set(zip(comp.tolist(), labels.tolist()))) == k  # the components, up to a permutation


@pytest.mark.parametrize("p", [1.5, 1.2])
def test_p_below_2_stage_stops_on_the_optimum(p):
    """Started on the component span, every difference inside a component is
    a tie: the gradient is exactly zero and the stage takes no step."""
    g, comp = components_graph([30, 24, 36], 3)
    ind = np.zeros((g.n, 3))
    ind[np.arange(g.n), comp] = 1.0
    U, st = oracle.rtr_newton(g, oracle.qf(ind), p, oracle.SolveOptions())
    assert st["outer"] == 0 and st["gnorm"] == 0.0 and oracle.objective(g, U, p) == 0.0


def test_p_below_2_solve_ends_with_zero_rcut_on_components():
    """The whole solve below p = 2 (two stages, k-means, RCut) from a
    perturbed indicator block: the components, and RCut = 0 (no edge cut)."""
    g, comp = components_graph([30, 24, 36], 3)
    k = 3
    ind = np.zeros((g.n, k))
    ind[np.arange(g.n), comp] = 1.0
    U0 = oracle.qf(ind + 0.2 * np.random.default_rng(7).standard_normal(ind.shape))
    U, labels, rc, stages = oracle.solve(g, U0, (1.6, 1.3), oracle.SolveOptions(max_outer=60))
    assert rc == 0.0
    assert len(set(zip(comp.tolist(), labels.tolist()))) == k
    assert stages[0]["f"] <= 1e-12 * oracle.objective(g, U0, 1.6)


def test_p_below_2_newton_converges_quadratically():
    """Near a minimiser where no difference vanishes, F_p is smooth and
    Riemannian Newton with the exact Hessian converges quadratically (Absil,
    Mahony & Sepulchre, Thm. 7.4.11; truncated CG stops at ||r|| <=
    ||g||^(1 + theta), theta = 1): once ||grad|| is below 1e-6 of its start
    it reaches 1e-12 within three steps.  Algorithm 1's form, which leaves out
    the quotient's rank-two terms, is not the Hessian of F_p, and from the same
    start it converges only linearly (not below 1e-8 in 80 steps)."""
    g = wl.sbm_sampled(np.random.default_rng(3), 150, 3, 8.0, 0.85, np.float64)
    k = 3
    U2, _ = oracle.rtr_newton(g, wl.orthonormal_block(3, g.n, k, np.float64), 2.0,
                              oracle.SolveOptions(max_outer=60, gtol_rel=1e-12))
    U, st = oracle.rtr_newton(g, U2, 1.5, oracle.SolveOptions(max_outer=80, gtol_rel=1e-12))
    h = np.array(st["history"]) / st["gnorm0"]
    assert h[-1] <= 1e-12
    first = int(np.argmax(h <= 1e-6))
    assert h[first] <= 1e-6 and len(h) - 1 - first <= 3, h[-8:]
    _, sta = oracle.rtr_newton(g, U2, 1.5, oracle.SolveOptions(max_outer=80, gtol_rel=1e-12, hessian="alg1"))
    assert min(sta["history"]) / sta["gnorm0"] > 1e-8
