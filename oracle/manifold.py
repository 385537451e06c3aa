"""Riemannian Newton with truncated CG on the Grassmann manifold, in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Section 2) minimises Eq. 1 on the Grassmann manifold with Newton's
method, one solve per p with p lowered stage by stage toward 1, and solves the
Newton subproblems by truncated conjugate gradients (in ROPTLIB, given the
Euclidean gradient and Hessian-vector product).  It prints no further detail, so the following readings are
taken, each the textbook form (Absil, Mahony & Sepulchre, "Optimization
Algorithms on Matrix Manifolds", 2008: the Riemannian trust-region method and
its Steihaug-Toint truncated CG; Edelman, Arias & Smith 1998 for the
Grassmann geometry):

  * metric: <A, B> = trace(A^T B) on n x k blocks;
  * tangent projection: P_U(G) = G - U (U^T G);
  * Riemannian gradient: P_U(grad F);
  * Riemannian Hessian: Hess[eta] = P_U(H eta) - eta (U^T grad F);
  * retraction: R_U(eta) = qf(U + eta), the Q of a thin QR with diag(R) > 0;
  * outer method: trust-region Newton (radius update 1/4 and 3/4 rules,
    acceptance when rho > rho_prime and the model decreased), with the
    ratio rho regularised by rho_reg * max(1, |f|) on both sides;
  * Euclidean Hessian: the exact Hessian of the quotient N/D by default;
    optionally (hessian="alg1") only the sparse-plus-diagonal matrix that
    Algorithm 1 applies, without the quotient's rank-two terms;
  * inner method: Steihaug-Toint truncated CG from eta = 0 without a
    preconditioner, stopping on negative curvature, on reaching the radius,
    when ||r|| <= ||r_0|| min(||r_0||^theta, kappa), or after max_inner steps;
    <eta, delta> and <delta, delta> follow their CG recurrences;
  * continuation: each p of the schedule is solved in turn, warm started from
    the previous stage's U.
F_p is not invariant under U -> UQ for p < 2; the projection and retraction
above are used as stated all the same (the paper's Grassmann formulation).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import plap
from .cluster import kmeans, rcut


@dataclasses.dataclass
class SolveOptions:
    """Options of the trust-region Newton solve; the CUDA library's options
    struct carries the same fields with the same defaults."""

    max_outer: int = 30          # Newton steps per value of p
    max_inner: int = 50          # truncated-CG steps per Newton step
    gtol_rel: float = 1e-6       # stop when ||grad|| <= gtol_rel ||grad at stage start||
    gtol_abs: float = 0.0        # ... or when ||grad|| <= gtol_abs
    theta: float = 1.0           # tCG superlinear exponent
    kappa: float = 0.1           # tCG linear factor
    delta_bar_scale: float = 1.0  # Delta_bar = scale * sqrt(k)
    delta0_scale: float = 0.1    # Delta_0 = scale * Delta_bar
    rho_prime: float = 0.1       # acceptance threshold
    rho_reg: float = 1e-10       # regularisation of rho, relative to max(1, |f|)
    kmeans_restarts: int = 10
    kmeans_max_iter: int = 300
    seed: int = 0
    # "exact": the Hessian of the quotient N/D (sparse + diagonal + rank-two
    # terms); "alg1": only the sparse-plus-diagonal matrix Algorithm 1 applies
    hessian: str = "exact"


def inner(A, B):
    """<A, B> = trace(A^T B)."""
    return float(np.sum(np.asarray(A) * np.asarray(B)))


def project(U, G):
    """Tangent projection P_U(G) = G - U (U^T G)."""
    return G - U @ (U.T @ G)


def riemannian_hessian(U, egrad, ehv, eta):
    """Hess[eta] = P_U(H eta) - eta (U^T grad F)."""
    return project(U, ehv) - eta @ (U.T @ egrad)


def qf(A):
    """Q factor of the thin QR of A, signs chosen so that diag(R) > 0."""
    q, r = np.linalg.qr(A)
    return q * np.where(np.diag(r) < 0, -1.0, 1.0)


def tcg(hess, grad, Delta, theta, kappa, max_inner):
    """Steihaug-Toint truncated CG for min <grad,eta> + 1/2 <eta, Hess eta>,
    ||eta|| <= Delta.  Returns (eta, Hess eta, iterations, reason, on_boundary)
    with reason in {"negative_curvature", "radius", "converged", "max_inner"}."""
    eta = np.zeros_like(grad)
    Heta = np.zeros_like(grad)
    r = grad.copy()
    r_r = inner(r, r)
    norm_r0 = math.sqrt(r_r)
    delta = -r
    e_Pe = 0.0      # <eta, eta>
    e_Pd = 0.0      # <eta, delta>
    d_Pd = r_r      # <delta, delta>
    for j in range(1, max_inner + 1):
        Hdelta = hess(delta)
        d_Hd = inner(delta, Hdelta)
        alpha = r_r / d_Hd if d_Hd != 0.0 else math.inf
        e_Pe_new = e_Pe + 2.0 * alpha * e_Pd + alpha * alpha * d_Pd
        if d_Hd <= 0.0 or e_Pe_new >= Delta * Delta:
            tau = (-e_Pd + math.sqrt(e_Pd * e_Pd + d_Pd * (Delta * Delta - e_Pe))) / d_Pd
            eta = eta + tau * delta
            Heta = Heta + tau * Hdelta
            return eta, Heta, j, ("negative_curvature" if d_Hd <= 0.0 else "radius"), True
        e_Pe = e_Pe_new
        eta = eta + alpha * delta
        Heta = Heta + alpha * Hdelta
        r = r + alpha * Hdelta
        r_r_old = r_r
        r_r = inner(r, r)
        if math.sqrt(r_r) <= norm_r0 * min(norm_r0 ** theta, kappa):
            return eta, Heta, j, "converged", False
        beta = r_r / r_r_old
        delta = -r + beta * delta
        e_Pd = beta * (e_Pd + alpha * d_Pd)
        d_Pd = r_r + beta * beta * d_Pd
    return eta, Heta, max_inner, "max_inner", False


def rtr_newton(g, U, p, opts: SolveOptions):
    """Trust-region Newton on Gr(k, n) for F_p at fixed p, from U.

    Returns (U, stats) with stats a dict: outer, inner, f, gnorm, gnorm0 and
    history, the ||rg|| of the iterate after each Newton step.
    """
    k = U.shape[1]
    Delta_bar = opts.delta_bar_scale * math.sqrt(k)
    Delta = opts.delta0_scale * Delta_bar

    def value_grad(X):
        return plap.objective(g, X, p), plap.euclidean_grad(g, X, p)

    f, egrad = value_grad(U)
    rg = project(U, egrad)
    gnorm = math.sqrt(inner(rg, rg))
    gnorm0 = gnorm
    outer = 0
    inner_total = 0
    history = []
    while outer < opts.max_outer:
        if gnorm <= max(opts.gtol_abs, opts.gtol_rel * gnorm0):
            break
        outer += 1

        ehvp = plap.alg1_sparse_hvp if opts.hessian == "alg1" else plap.euclidean_hvp

        def hess(eta, U=U, egrad=egrad):
            return riemannian_hessian(U, egrad, ehvp(g, U, eta, p), eta)

        eta, Heta, its, _reason, on_boundary = tcg(hess, rg, Delta, opts.theta,
                                                   opts.kappa, opts.max_inner)
        inner_total += its
        U_new = qf(U + eta)
        f_new = plap.objective(g, U_new, p)
        reg = opts.rho_reg * max(1.0, abs(f))
        num = f - f_new + reg
        den = -(inner(rg, eta) + 0.5 * inner(eta, Heta)) + reg
        model_decreased = den >= 0.0
        rho = num / den if den != 0.0 else -math.inf
        if (not model_decreased) or rho < 0.25 or math.isnan(rho):
            Delta = 0.25 * Delta
        elif rho > 0.75 and on_boundary:
            Delta = min(2.0 * Delta, Delta_bar)
        if model_decreased and rho > opts.rho_prime:
            U = U_new
            f, egrad = value_grad(U)
            rg = project(U, egrad)
            gnorm = math.sqrt(inner(rg, rg))
        history.append(gnorm)
    return U, dict(outer=outer, inner=inner_total, f=f, gnorm=gnorm, gnorm0=gnorm0,
                   delta=Delta, history=history)


def solve(g, U0, p_schedule, opts: SolveOptions | None = None, n_clusters=None):
    """p continuation + k-means + RCut.  Returns (U, labels, rcut, stats)."""
    opts = opts or SolveOptions()
    U = np.array(U0, dtype=np.float64)
    stages = []
    for p in p_schedule:
        U, st = rtr_newton(g, U, float(p), opts)
        st["p"] = float(p)
        stages.append(st)
    C = U.shape[1] if n_clusters is None else n_clusters
    labels, _centers, _inertia = kmeans(U, C, opts.seed, opts.kmeans_restarts, opts.kmeans_max_iter)
    return U, labels, rcut(g, labels, C), stages
