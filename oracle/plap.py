"""Objective, p-Laplacian, gradient and Hessian-vector product in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definitions followed (paper, Section 2):
  * Eq. 1:  F_p(U) = sum_l sum_{i,j} w_ij |u_i^l - u_j^l|^p / (2 ||u^l||_p^p),
    the double sum over ordered pairs of a symmetric W, so with both CSR
    triangles stored every undirected edge counts once after the 1/2.
  * p-Laplacian: (Delta_p u)_i = sum_j w_ij phi_p(u_i - u_j).
  * phi_p(x) = |x|^(p-1) sign(x), sign(0) = 0, so phi_p(0) = 0.
  * p-norm: ||u||_p^p = sum_i |u_i|^p, per column (the paper's "u in R" is
    read as u in R^n).

The paper does not print the gradient (EucGrad) or the Hessian it hands to
Algorithm 1.  Writing F_p = sum_l N_l / D_l with N_l = (1/2) sum_ij w_ij
|d_ij|^p and D_l = ||u^l||_p^p, the derivatives are:
  * grad N = p Delta_p u          (W symmetric, phi_p odd)
  * grad D = p phi_p(u)
  * grad f = (p / D) (Delta_p u - lambda phi_p(u)),  lambda = N / D
  * (Hess N eta)_a = p(p-1) sum_j w_aj |d_aj|^(p-2) (eta_a - eta_j)
  * (Hess D eta)_a = p(p-1) |u_a|^(p-2) eta_a
  * H eta = (Hess N eta - lambda Hess D eta) / D
            - (g_N <g_D,eta> + g_D <g_N,eta> - 2 lambda g_D <g_D,eta>) / D^2
    with g_N = grad N, g_D = grad D: the exact Hessian of the quotient.
Reading for p < 2 where |x|^(p-2) is unbounded: the edge term is 0 when
d_ij == 0 exactly and the vertex term is 0 when u_a == 0 exactly (the paper
applies no smoothing; a zero difference is treated as a zero-curvature edge).
At p = 2, |x|^0 = 1 everywhere, so the Hessian of N is exactly 2L (the
p-Laplacian at p = 2 is the graph Laplacian) even where values tie.

Graphs are any object with integer ``n`` and CSR arrays ``rowptr``, ``col``
and ``val`` holding both triangles of W.  Blocks U, V are n x k arrays.
"""
from __future__ import annotations

import numpy as np


def edge_list(g):
    """(row, col, weight) of every stored entry of W, in CSR order, float64."""
    rowptr = np.asarray(g.rowptr, dtype=np.int64)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rowptr))
    return rows, np.asarray(g.col, dtype=np.int64), np.asarray(g.val, dtype=np.float64)


def phi_p(x, p):
    """phi_p(x) = |x|^(p-1) sign(x) (Section 2), with sign(0) = 0."""
    x = np.asarray(x, dtype=np.float64)
    return np.abs(x) ** (p - 1.0) * np.sign(x)


def abs_pow_pm2(x, p):
    """|x|^(p-2); for p < 2 read as 0 where x == 0 (the zero-curvature
    reading), for p = 2 identically 1."""
    x = np.asarray(x, dtype=np.float64)
    if p == 2.0:
        return np.ones_like(x)
    out = np.zeros_like(x)
    nz = x != 0
    out[nz] = np.abs(x[nz]) ** (p - 2.0)
    return out


def p_norm_p(U, p):
    """||u^l||_p^p = sum_i |u_i^l|^p for every column l (Section 2)."""
    return np.sum(np.abs(np.asarray(U, dtype=np.float64)) ** p, axis=0)


def _columns(U):
    U = np.asarray(U, dtype=np.float64)
    return U[:, None] if U.ndim == 1 else U


def _row_sum(rows, terms, n):
    """out[i, l] = sum of terms[e, l] over the entries e of row i."""
    out = np.zeros((n, terms.shape[1]))
    for l in range(terms.shape[1]):
        out[:, l] = np.bincount(rows, weights=terms[:, l], minlength=n)
    return out


def objective_parts(g, U, p):
    """(N, D) per column: N_l = 1/2 sum_ij w_ij |u_i - u_j|^p, D_l = ||u^l||_p^p."""
    U = _columns(U)
    rows, col, w = edge_list(g)
    d = U[rows] - U[col]
    N = 0.5 * np.sum(w[:, None] * np.abs(d) ** p, axis=0)
    return N, p_norm_p(U, p)


def objective(g, U, p):
    """F_p(U) of Eq. 1."""
    N, D = objective_parts(g, U, p)
    return float(np.sum(N / D))


def p_laplacian(g, U, p):
    """(Delta_p u^l)_i = sum_j w_ij phi_p(u_i^l - u_j^l), all columns."""
    U = _columns(U)
    rows, col, w = edge_list(g)
    return _row_sum(rows, w[:, None] * phi_p(U[rows] - U[col], p), g.n)


def euclidean_grad(g, U, p):
    """Euclidean gradient of F_p: column l is (p/D_l)(Delta_p u^l - lambda_l phi_p(u^l))."""
    U = _columns(U)
    N, D = objective_parts(g, U, p)
    lam = N / D
    return (p / D) * (p_laplacian(g, U, p) - lam * phi_p(U, p))


def euclidean_hvp(g, U, V, p):
    """Exact Euclidean Hessian of F_p applied to V (block diagonal over columns)."""
    U = _columns(U)
    V = _columns(V)
    rows, col, w = edge_list(g)
    N, D = objective_parts(g, U, p)
    lam = N / D
    c = p * (p - 1.0)
    sparse = c * _row_sum(rows, w[:, None] * abs_pow_pm2(U[rows] - U[col], p)
                          * (V[rows] - V[col]), g.n)
    vertex = c * abs_pow_pm2(U, p) * V
    gN = p * p_laplacian(g, U, p)
    gD = p * phi_p(U, p)
    cN = np.sum(gN * V, axis=0)
    cD = np.sum(gD * V, axis=0)
    return (sparse - lam * vertex) / D - (gN * cD + gD * cN - 2.0 * lam * gD * cD) / D ** 2


def alg1_sparse_hvp(g, U, V, p):
    """Algorithm 1 applied to the sparse-plus-diagonal part of the Hessian.

    For every column l the matrix Hc^l = (Hess N - lambda Hess D)/D is split
    as in Algorithm 1's inputs, D[l] = diag(Hc^l) and H[l] = diag(Hc^l) - Hc^l
    (W's pattern), and the column result is r_l = D[l] o eta_l - eta_l H[l].
    The rank-two terms of the quotient's Hessian are not part of this form.
    """
    U = _columns(U)
    V = _columns(V)
    rows, col, w = edge_list(g)
    N, D = objective_parts(g, U, p)
    lam = N / D
    c = p * (p - 1.0)
    out = np.zeros_like(V)
    for l in range(U.shape[1]):
        off = c * w * abs_pow_pm2(U[rows, l] - U[col, l], p) / D[l]   # entries of H[l]
        diag = (np.bincount(rows, weights=off, minlength=g.n)
                - lam[l] * c * abs_pow_pm2(U[:, l], p) / D[l])        # D[l]
        v = np.bincount(rows, weights=off * V[col, l], minlength=g.n)  # vxm(eta_l, H[l])
        out[:, l] = diag * V[:, l] - v                                 # D[l] o eta_l - v
    return out
