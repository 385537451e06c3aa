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
