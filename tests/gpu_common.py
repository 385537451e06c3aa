"""Shared helpers of the GPU parity tests (graphs, tolerances, comparisons)."""
import numpy as np

from paper_2605_26975_gb300 import workloads as wl

# Tolerances: F and the gradient within 1e-5 relative, the Hessian-vector
# product within 1e-4 relative (per column, Frobenius), for the FP32 path;
# the FP64 plain path within 1e-11.
TOL_F = 1e-5
TOL_GRAD = 1e-5
TOL_HVP = 1e-4
TOL_F64 = 1e-11


def rel_col(a, b):
    """max over columns of ||a_l - b_l|| / ||b_l||."""
    a = np.asarray(a, dtype=np.float64).reshape(b.shape)
    num = np.linalg.norm(a - b, axis=0)
    den = np.linalg.norm(b, axis=0)
    den = np.where(den == 0, 1.0, den)
    return float(np.max(num / den))


def star_plus_powerlaw(seed=3, n=20_000):
    """Degree-corrected SBM with Pareto propensities (hub rows) plus one star
    centre joined to a tenth of the vertices: exercises the split of long rows."""
    g = wl.dcsbm_powerlaw(seed, n=n, blocks=4, mean_degree=12.0)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    a = np.concatenate([rows, np.zeros(n // 10, dtype=np.int64)])
    b = np.concatenate([g.col.astype(np.int64), np.arange(1, n // 10 + 1)])
    w = np.concatenate([g.val.astype(np.float64), np.full(n // 10, 0.5)])
    keep = a < b
    return wl.csr_from_undirected(n, a[keep], b[keep], w[keep])


def with_isolated(seed=4, n=3000):
    """SBM with about 5% of the vertices left isolated (empty rows)."""
    rng = np.random.default_rng(seed)
    g = wl.sbm_sampled(rng, n, 4, 10.0, 0.9)
    iso = rng.random(n) < 0.05
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    keep = (~iso[rows]) & (~iso[g.col]) & (rows < g.col)
    return wl.csr_from_undirected(n, rows[keep], g.col[keep], g.val[keep])


def small_graphs():
    return {
        "sbm": wl.sbm_sampled(np.random.default_rng(1), 3001, 4, 14.0, 0.85),
        "grid": wl.grid3d_longrange(2, side=13, frac_long=0.01),
        "knn": wl.knn_gaussian_mixture(5, n=4000, mixtures=4),
        "hubs": star_plus_powerlaw(),
        "isolated": with_isolated(),
    }


def rel_terms(a, ref, scale):
    """max over columns of ||a_l - ref_l|| / ||scale_l||, with `scale` the
    elementwise sum of the magnitudes of the terms that make up ref.  This is
    the rounding bound of a sum of terms: it stays meaningful where the terms
    cancel (a column of a tiny graph near a stationary point)."""
    a = np.asarray(a, dtype=np.float64).reshape(ref.shape)
    num = np.linalg.norm(a - ref, axis=0)
    den = np.linalg.norm(scale, axis=0)
    den = np.where(den == 0, 1.0, den)
    return float(np.max(num / den))


def grad_term_scale(oracle, g, U, p):
    """|(p/D)(Delta_p u)| + |(p/D) lambda phi_p(u)| term by term."""
    rows, col, w = oracle.edge_list(g)
    N, D = oracle.objective_parts(g, U, p)
    out = np.zeros_like(U)
    for l in range(U.shape[1]):
        d = np.abs(U[rows, l] - U[col, l])
        dabs = np.bincount(rows, weights=w * d ** (p - 1.0), minlength=g.n)
        out[:, l] = (p / D[l]) * (dabs + (N[l] / D[l]) * np.abs(U[:, l]) ** (p - 1.0))
    return out


def rel_elem(a, ref, scale):
    """max over entries of |a - ref| / scale, with `scale` the magnitude of the
    terms that make up ref (an entry whose scale is 0 must match exactly)."""
    a = np.asarray(a, dtype=np.float64).reshape(ref.shape)
    err = np.abs(a - ref)
    zero = scale == 0
    if np.any(err[zero] != 0):
        return float("inf")
    return float(np.max(np.where(zero, 0.0, err / np.where(zero, 1.0, scale)), initial=0.0))


def tied_heavy_graph(seed=12, n=3000):
    """SBM with weights log-uniform in [1, 1e6]: with quantised blocks many
    entries tie (u_i == u_j) under a weight far above 2^(128 - 126 (2 - p)),
    the size at which w 2^(126 (2 - p)) leaves the FP32 range for p near 1."""
    rng = np.random.default_rng(seed)
    g = wl.sbm_sampled(rng, n, 4, 12.0, 0.85)
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    keep = rows < g.col
    a, b = rows[keep], g.col[keep].astype(np.int64)
    w = 10.0 ** rng.uniform(0.0, 6.0, a.size)
    return wl.csr_from_undirected(n, a, b, w)


def quantised_block(seed, n, k):
    """Values in {-0.75, -0.5, ..., 0.75}: many exact ties and exact zeros."""
    rng = np.random.default_rng(seed)
    return (rng.integers(-3, 4, size=(n, k)) * 0.25).astype(np.float32)


def hvp_term_scale(oracle, g, U, V, p):
    """Magnitudes of the terms of the exact Hessian product: the sparse part,
    the diagonal part and the three rank-two terms, added term by term (the
    column dots <g_D, v>, <g_N, v> as sums of the magnitudes of their terms,
    which is what bounds their rounding)."""
    rows, col, w = oracle.edge_list(g)
    N, D = oracle.objective_parts(g, U, p)
    c = p * (p - 1.0)
    out = np.zeros_like(U)
    for l in range(U.shape[1]):
        u, v = U[:, l], V[:, l]
        lam = N[l] / D[l]
        s = np.bincount(rows, weights=c * w * oracle.abs_pow_pm2(u[rows] - u[col], p)
                        * np.abs(v[rows] - v[col]), minlength=g.n)
        diag = lam * c * oracle.abs_pow_pm2(u, p) * np.abs(v)
        gN = p * oracle.p_laplacian(g, U[:, l:l + 1], p)[:, 0]
        gD = p * oracle.phi_p(u, p)
        aDv, aNv = np.abs(gD) @ np.abs(v), np.abs(gN) @ np.abs(v)
        r2 = (np.abs(gN) * aDv + np.abs(gD) * aNv + 2 * lam * np.abs(gD) * aDv) / D[l] ** 2
        out[:, l] = (s + diag) / D[l] + r2
    return out


def check_eval(api, g, G, U, p):
    """pspec_eval on U (FP32) against the oracle: F, N, D, and the gradient
    per column and entry by entry."""
    import torch
    import oracle
    Ud = torch.from_numpy(U).cuda()
    F, grad, parts = G.eval(Ud, p, parts=True)
    torch.cuda.synchronize()
    assert G.status() == 0
    U64 = U.astype(np.float64)
    F_ref = oracle.objective(g, U64, p)
    N, D = oracle.objective_parts(g, U64, p)
    gr_ref = oracle.euclidean_grad(g, U64, p)
    assert abs(F.item() - F_ref) <= TOL_F * abs(F_ref)
    P = parts.cpu().numpy()
    k = U.shape[1]
    assert np.allclose(P[:k], N, rtol=TOL_F, atol=0)
    assert np.allclose(P[k:], D, rtol=TOL_F, atol=0)
    got = grad.cpu().numpy()
    assert rel_col(got, gr_ref) <= TOL_GRAD
    # entry by entry, against the magnitude of the entry's terms: a wrong
    # value on a low-degree or small-|u| row cannot hide in a column norm
    assert rel_elem(got, gr_ref, grad_term_scale(oracle, g, U64, p)) <= TOL_GRAD


def check_hvp(api, g, G, U, V, p):
    """pspec_hvp on U, V (FP32) against the oracle, per column and entry by
    entry."""
    import torch
    import oracle
    Ud = torch.from_numpy(U).cuda()
    Vd = torch.from_numpy(V).cuda()
    HV = G.hvp(Ud, Vd, p)
    torch.cuda.synchronize()
    assert G.status() == 0
    U64, V64 = U.astype(np.float64), V.astype(np.float64)
    ref = oracle.euclidean_hvp(g, U64, V64, p)
    got = HV.cpu().numpy()
    assert rel_col(got, ref) <= TOL_HVP
    assert rel_elem(got, ref, hvp_term_scale(oracle, g, U64, V64, p)) <= TOL_HVP
