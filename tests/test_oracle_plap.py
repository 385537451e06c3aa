"""Pins of the FP64 oracle's objective, p-Laplacian, gradient and Hessian.

Each check ties the oracle to something other than its own formula: closed
forms on tiny graphs, the p = 2 reduction to the dense graph Laplacian,
brute-force double loops over a dense W, invariances of Eq. 1, and central
finite differences with Richardson extrapolation.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_26975_gb300 import workloads as wl

PS = [2.0, 1.8, 1.5, 1.3, 1.1]


def dense_graph(Wd):
    """CSR of a dense symmetric matrix (zero diagonal)."""
    n = Wd.shape[0]
    iu, ju = np.nonzero(np.triu(Wd, 1))
    return wl.csr_from_undirected(n, iu, ju, Wd[iu, ju], np.float64)


def random_dense_w(rng, n, density=0.4):
    A = np.triu((rng.random((n, n)) < density) * rng.uniform(0.2, 2.0, (n, n)), 1)
    return A + A.T


def laplacian(Wd):
    return np.diag(Wd.sum(axis=1)) - Wd


# ----------------------------------------------------------------- phi_p

@pytest.mark.parametrize("p", PS)
def test_phi_basic(p):
    assert oracle.phi_p(0.0, p) == 0.0
    x = np.array([-3.5, -0.25, 1e-7, 0.8, 12.0])
    assert np.allclose(oracle.phi_p(-x, p), -oracle.phi_p(x, p), rtol=0, atol=0)
    for xi in x:
        assert math.isclose(abs(oracle.phi_p(xi, p)), math.pow(abs(xi), p - 1), rel_tol=1e-15)


def test_phi_exact_values():
    assert oracle.phi_p(4.0, 1.5) == 2.0
    assert oracle.phi_p(-9.0, 1.5) == -3.0
    assert np.array_equal(oracle.phi_p(np.array([-2.5, 0.0, 3.0]), 2.0), np.array([-2.5, 0.0, 3.0]))


# ------------------------------------------------------------- objective

@pytest.mark.parametrize("p", PS)
def test_two_vertex_closed_form(p):
    w = 0.7
    g = dense_graph(np.array([[0.0, w], [w, 0.0]]))
    assert math.isclose(oracle.objective(g, np.array([[1.0], [-1.0]]), p), 2 ** (p - 1) * w,
                        rel_tol=1e-14)
    a, b = 0.3, -1.7
    ref = w * abs(a - b) ** p / (abs(a) ** p + abs(b) ** p)
    assert math.isclose(oracle.objective(g, np.array([[a], [b]]), p), ref, rel_tol=1e-14)
    # derivative of the two-variable closed form
    den = abs(a) ** p + abs(b) ** p
    s = math.copysign(1.0, a - b)
    da = w * (p * abs(a - b) ** (p - 1) * s * den - abs(a - b) ** p * p * abs(a) ** (p - 1)
              * math.copysign(1.0, a)) / den ** 2
    db = w * (-p * abs(a - b) ** (p - 1) * s * den - abs(a - b) ** p * p * abs(b) ** (p - 1)
              * math.copysign(1.0, b)) / den ** 2
    gr = oracle.euclidean_grad(g, np.array([[a], [b]]), p)
    assert np.allclose(gr[:, 0], [da, db], rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", PS)
def test_two_level_vector(p):
    rng = np.random.default_rng(5)
    n = 30
    Wd = random_dense_w(rng, n)
    g = dense_graph(Wd)
    A = rng.random(n) < 0.4
    a, b = 1.3, -0.6
    u = np.where(A, a, b)
    cut = sum(Wd[i, j] for i in range(n) for j in range(n) if A[i] and not A[j])
    ref = cut * abs(a - b) ** p / (A.sum() * abs(a) ** p + (~A).sum() * abs(b) ** p)
    assert math.isclose(oracle.objective(g, u, p), ref, rel_tol=1e-13)
    lap = oracle.p_laplacian(g, u, p)[:, 0]
    for i in range(n):
        other = sum(Wd[i, j] for j in range(n) if A[j] != A[i])
        expect = (abs(a - b) ** (p - 1)) * (1 if A[i] else -1) * other
        assert math.isclose(lap[i], expect, rel_tol=1e-13, abs_tol=1e-15)


@pytest.mark.parametrize("p", PS)
def test_component_indicators_zero(p):
    rng = np.random.default_rng(1)
    blocks = [random_dense_w(rng, m, 0.7) for m in (5, 7, 4)]
    n = sum(b.shape[0] for b in blocks)
    Wd = np.zeros((n, n))
    U = np.zeros((n, 3))
    o = 0
    for c, B in enumerate(blocks):
        m = B.shape[0]
        Wd[o:o + m, o:o + m] = B
        U[o:o + m, c] = rng.uniform(0.5, 2.0)
        o += m
    g = dense_graph(Wd)
    assert oracle.objective(g, U, p) == 0.0


@pytest.mark.parametrize("p", PS)
def test_scale_and_permutation_invariance(p):
    rng = np.random.default_rng(2)
    n, k = 25, 3
    Wd = random_dense_w(rng, n)
    g = dense_graph(Wd)
    U = rng.standard_normal((n, k))
    f = oracle.objective(g, U, p)
    c = np.array([2.5, -0.3, 7.0])
    assert math.isclose(oracle.objective(g, U * c, p), f, rel_tol=1e-13)
    perm = rng.permutation(n)
    gp = dense_graph(Wd[np.ix_(perm, perm)])
    assert math.isclose(oracle.objective(gp, U[perm], p), f, rel_tol=1e-13)


def test_p2_is_rayleigh_quotient_and_laplacian():
    rng = np.random.default_rng(3)
    n, k = 20, 4
    Wd = random_dense_w(rng, n)
    g = dense_graph(Wd)
    L = laplacian(Wd)
    U = rng.standard_normal((n, k))
    ref = sum(U[:, l] @ L @ U[:, l] / (U[:, l] @ U[:, l]) for l in range(k))
    assert math.isclose(oracle.objective(g, U, 2.0), ref, rel_tol=1e-13)
    assert np.allclose(oracle.p_laplacian(g, U, 2.0), L @ U, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("p", PS)
def test_brute_force_double_loop(p):
    rng = np.random.default_rng(4)
    n, k = 12, 2
    Wd = random_dense_w(rng, n, 0.5)
    g = dense_graph(Wd)
    U = rng.standard_normal((n, k))
    N, D = oracle.objective_parts(g, U, p)
    for l in range(k):
        nb = 0.0
        lap = np.zeros(n)
        for i in range(n):
            for j in range(n):
                if Wd[i, j] != 0:
                    dd = U[i, l] - U[j, l]
                    nb += Wd[i, j] * abs(dd) ** p
                    lap[i] += Wd[i, j] * math.copysign(abs(dd) ** (p - 1), dd)
        db = sum(abs(U[i, l]) ** p for i in range(n))
        assert math.isclose(N[l], nb / 2, rel_tol=1e-13)
        assert math.isclose(D[l], db, rel_tol=1e-13)
        got = oracle.p_laplacian(g, U[:, l], p)[:, 0]
        assert np.allclose(got, lap, rtol=1e-13, atol=1e-14)
        # <Delta_p u, u> = N  (antisymmetry of phi_p(u_i - u_j) under i <-> j)
        assert math.isclose(float(got @ U[:, l]), nb / 2, rel_tol=1e-12)


@pytest.mark.parametrize("p", PS)
def test_laplacian_homogeneity(p):
    rng = np.random.default_rng(6)
    g = dense_graph(random_dense_w(rng, 15))
    u = rng.standard_normal(15)
    for c in (3.0, -0.5):
        lhs = oracle.p_laplacian(g, c * u, p)
        rhs = abs(c) ** (p - 2) * c * oracle.p_laplacian(g, u, p)
        assert np.allclose(lhs, rhs, rtol=1e-13, atol=1e-14)


# -------------------------------------------------------------- gradient

def richardson(fun, h):
    d1 = fun(h)
    d2 = fun(h / 2)
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("p", PS)
def test_gradient_finite_differences(p):
    rng = np.random.default_rng(7)
    n, k = 10, 2
    g = dense_graph(random_dense_w(rng, n, 0.6))
    # well separated values keep the stencil away from the kink of |d|^p
    U = rng.permutation(n)[:, None] * 0.29 + np.array([[0.07, -0.4]]) + 0.01 * rng.random((n, k))
    U = U - U.mean(axis=0) + 0.017
    G = oracle.euclidean_grad(g, U, p)
    fd = np.zeros_like(U)
    for i in range(n):
        for l in range(k):
            E = np.zeros_like(U)
            E[i, l] = 1.0
            fd[i, l] = richardson(lambda h: (oracle.objective(g, U + h * E, p)
                                             - oracle.objective(g, U - h * E, p)) / (2 * h), 1e-4)
    assert np.allclose(G, fd, rtol=1e-7, atol=1e-9 * np.abs(G).max())


@pytest.mark.parametrize("p", PS)
def test_gradient_euler_and_homogeneity(p):
    rng = np.random.default_rng(8)
    n, k = 40, 3
    g = dense_graph(random_dense_w(rng, n, 0.2))
    U = rng.standard_normal((n, k))
    G = oracle.euclidean_grad(g, U, p)
    for l in range(k):
        assert abs(G[:, l] @ U[:, l]) <= 1e-13 * np.linalg.norm(G[:, l]) * np.linalg.norm(U[:, l])
    c = np.array([3.0, -2.0, 0.5])
    assert np.allclose(oracle.euclidean_grad(g, U * c, p), G / c, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ HVP

@pytest.mark.parametrize("p", PS)
def test_hvp_finite_differences(p):
    rng = np.random.default_rng(9)
    n, k = 14, 2
    g = dense_graph(random_dense_w(rng, n, 0.5))
    # well separated values: no edge difference crosses zero inside the stencil
    U = rng.permutation(n)[:, None] * 0.37 + np.array([[0.11, -0.05]]) + 0.01 * rng.random((n, k))
    U = U - U.mean(axis=0) + 0.013
    V = rng.standard_normal((n, k))
    H = oracle.euclidean_hvp(g, U, V, p)
    fd = richardson(lambda h: (oracle.euclidean_grad(g, U + h * V, p)
                               - oracle.euclidean_grad(g, U - h * V, p)) / (2 * h), 1e-4)
    assert np.allclose(H, fd, rtol=1e-6, atol=1e-8 * np.abs(H).max())


@pytest.mark.parametrize("p", PS)
def test_hvp_euler_and_symmetry(p):
    rng = np.random.default_rng(10)
    n, k = 50, 3
    g = dense_graph(random_dense_w(rng, n, 0.15))
    U = rng.standard_normal((n, k))
    G = oracle.euclidean_grad(g, U, p)
    # f is homogeneous of degree 0 in each column, so H u = -grad f
    assert np.allclose(oracle.euclidean_hvp(g, U, U, p), -G, rtol=1e-11, atol=1e-12 * np.abs(G).max())
    X = rng.standard_normal((n, k))
    Y = rng.standard_normal((n, k))
    for l in range(k):
        a = oracle.euclidean_hvp(g, U, Y, p)[:, l] @ X[:, l]
        b = oracle.euclidean_hvp(g, U, X, p)[:, l] @ Y[:, l]
        assert math.isclose(a, b, rel_tol=1e-11, abs_tol=1e-12)


def test_hvp_p2_closed_form():
    rng = np.random.default_rng(11)
    n = 18
    Wd = random_dense_w(rng, n)
    g = dense_graph(Wd)
    L = laplacian(Wd)
    u = rng.standard_normal(n)
    eta = rng.standard_normal(n)
    D = u @ u
    lam = u @ L @ u / D
    ref = (2 / D) * (L @ eta - lam * eta) - (4 / D ** 2) * (
        (L @ u) * (u @ eta) + u * ((L @ u) @ eta) - 2 * lam * u * (u @ eta))
    assert np.allclose(oracle.euclidean_hvp(g, u, eta, 2.0)[:, 0], ref, rtol=1e-12, atol=1e-13)
    # Algorithm 1's sparse-plus-diagonal part at p = 2 is 2 (L - lambda I) / D
    assert np.allclose(oracle.alg1_sparse_hvp(g, u, eta, 2.0)[:, 0],
                       (2 / D) * (L @ eta - lam * eta), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("p", PS)
def test_alg1_plus_rank_two_is_exact_hessian(p):
    rng = np.random.default_rng(12)
    n, k = 30, 2
    g = dense_graph(random_dense_w(rng, n, 0.3))
    U = rng.standard_normal((n, k))
    V = rng.standard_normal((n, k))
    N, D = oracle.objective_parts(g, U, p)
    lam = N / D
    gN = p * oracle.p_laplacian(g, U, p)
    gD = p * oracle.phi_p(U, p)
    cN, cD = (gN * V).sum(0), (gD * V).sum(0)
    rank2 = (gN * cD + gD * cN - 2 * lam * gD * cD) / D ** 2
    assert np.allclose(oracle.alg1_sparse_hvp(g, U, V, p) - rank2,
                       oracle.euclidean_hvp(g, U, V, p), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("p", [1.5, 1.1])
def test_zero_difference_reading(p):
    # equal neighbouring values: that edge contributes no curvature (reading
    # for |d|^(p-2) at d == 0); a vertex value of 0 contributes no vertex term
    # Path 0 -(w=1)- 1 -(w=2)- 2 with u = (1/2, 1/2, -1): the edge 0-1 ties.
    # Worked by hand: N = 2 (3/2)^p, D = 2 (1/2)^p + 1, lambda = N / D,
    # g_N = p Delta_p u = (0, 2p (3/2)^(p-1), -2p (3/2)^(p-1)),
    # g_D = p phi_p(u) = (p h, p h, -p) with h = (1/2)^(p-1).
    g = dense_graph(np.array([[0, 1.0, 0], [1.0, 0, 2.0], [0, 2.0, 0]]))
    U = np.array([[0.5], [0.5], [-1.0]])
    c = p * (p - 1.0)
    N, D = 2 * 1.5 ** p, 2 * 0.5 ** p + 1
    lam = N / D
    h, t = 0.5 ** (p - 1), 1.5 ** (p - 1)
    gN = np.array([0.0, 2 * p * t, -2 * p * t])
    gD = np.array([p * h, p * h, -p])

    def expect(HNv, HDv, v):
        cN, cD = gN @ v, gD @ v
        return (HNv - lam * HDv) / D - (gN * cD + gD * cN - 2 * lam * gD * cD) / D ** 2

    # v = e_0: vertex 0's only edge ties, so the sparse part is 0 everywhere
    # (a clamped or regularised |0|^(p-2) would make it huge); the vertex term
    # is p(p-1) (1/2)^(p-2) at vertex 0.
    v = np.array([1.0, 0.0, 0.0])
    ref = expect(np.zeros(3), np.array([c * 0.5 ** (p - 2), 0, 0]), v)
    # the same entries expanded by hand
    assert np.allclose(ref, [-lam * c * 0.5 ** (p - 2) / D + 2 * lam * p * p * h * h / D ** 2,
                             -(2 * p * p * t * h - 2 * lam * p * p * h * h) / D ** 2,
                             (2 * p * p * t * h - 2 * lam * p * p * h) / D ** 2], rtol=1e-14)
    H = oracle.euclidean_hvp(g, U, v[:, None], p)[:, 0]
    assert np.allclose(H, ref, rtol=1e-13, atol=0)
    # v = e_1: only the untied edge 1-2 bends, 2 (3/2)^(p-2) (v_1 - v_2) at 1
    # and at 2 the mirror; the tie 0-1 adds nothing at 0 or 1
    v = np.array([0.0, 1.0, 0.0])
    s = 2 * 1.5 ** (p - 2)
    ref = expect(c * np.array([0.0, s, -s]), np.array([0, c * 0.5 ** (p - 2), 0]), v)
    H = oracle.euclidean_hvp(g, U, v[:, None], p)[:, 0]
    assert np.allclose(H, ref, rtol=1e-13, atol=0)
    # a zero vertex value: u = (0, 1/2, -1), v = e_0 gives no vertex term at 0
    # and phi_p(0) = 0 in g_D
    U0 = np.array([[0.0], [0.5], [-1.0]])
    assert oracle.abs_pow_pm2(np.array([0.0, 2.0]), p)[0] == 0.0
    assert oracle.phi_p(0.0, p) == 0.0
    H0 = oracle.euclidean_hvp(g, U0, np.array([[1.0], [0.0], [0.0]]), p)
    assert np.all(np.isfinite(H0))
    N0 = 0.5 ** p + 2 * 1.5 ** p
    D0 = 0.5 ** p + 1
    lam0 = N0 / D0
    gN0 = p * np.array([-(0.5 ** (p - 1)), 0.5 ** (p - 1) + 2 * t, -2 * t])
    gD0 = p * np.array([0.0, h, -1.0])
    HN0 = c * np.array([0.5 ** (p - 2), -(0.5 ** (p - 2)), 0.0])  # edge 0-1: |d| = 1/2
    cN0, cD0 = gN0[0], gD0[0]
    ref0 = (HN0 - lam0 * 0.0) / D0 - (gN0 * cD0 + gD0 * cN0 - 2 * lam0 * gD0 * cD0) / D0 ** 2
    assert np.allclose(H0[:, 0], ref0, rtol=1e-13, atol=1e-15)


def test_p2_hessian_with_ties_is_laplacian():
    # at p = 2 the sparse part of the Hessian is 2 L / D even where values tie
    rng = np.random.default_rng(13)
    n = 16
    Wd = random_dense_w(rng, n)
    g = dense_graph(Wd)
    L = laplacian(Wd)
    u = np.repeat([0.5, -0.25, 1.0, 0.0], 4)        # ties and zeros
    eta = rng.standard_normal(n)
    D = u @ u
    lam = u @ L @ u / D
    ref = (2 / D) * (L @ eta - lam * eta) - (4 / D ** 2) * (
        (L @ u) * (u @ eta) + u * ((L @ u) @ eta) - 2 * lam * u * (u @ eta))
    assert np.allclose(oracle.euclidean_hvp(g, u, eta, 2.0)[:, 0], ref, rtol=1e-12, atol=1e-13)
