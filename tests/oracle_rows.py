"""Oracle quantities of graphs too large for one whole-graph oracle call.

At the full workload sizes (8,000,000 vertices and 48M stored entries) a
single numpy call of the oracle would hold tens of GB of temporaries.  The
helpers below assemble the same quantities from the oracle's own functions
applied to pieces of the graph:

  * a row block: the rows r0..r1 of W as a graph on all n vertices (other
    rows empty), so objective_parts gives that block's share of N and
    p_laplacian that block's rows of Delta_p u;
  * a star: one vertex and its neighbours, with only the centre's row stored,
    so p_laplacian and alg1_sparse_hvp give the centre's row.

The per-column scalars are then combined by the quotient rule the oracle
itself uses (Section 2: grad = (p/D)(Delta_p u - lambda phi_p(u)), and the
exact Hessian of N/D).  tests/test_oracle_rows.py checks every helper
against the whole-graph oracle on small graphs.
"""
import numpy as np

import oracle
from paper_2605_26975_gb300 import workloads as wl


def row_chunk(g, r0, r1):
    """The rows r0..r1 of W as a graph on all n vertices (other rows empty)."""
    rp = np.clip(g.rowptr, g.rowptr[r0], g.rowptr[r1]) - g.rowptr[r0]
    rp[:r0] = 0
    rp[r1:] = rp[r1]
    e0, e1 = g.rowptr[r0], g.rowptr[r1]
    return wl.CSRGraph(g.n, rp, g.col[e0:e1], g.val[e0:e1])


def chunks(n, rows_per_chunk):
    for r0 in range(0, n, rows_per_chunk):
        yield r0, min(n, r0 + rows_per_chunk)


def oracle_N_D(g, U64, p, rows_per_chunk=400_000):
    """N_l (summed over row blocks) and D_l of every column."""
    N = np.zeros(U64.shape[1])
    for r0, r1 in chunks(g.n, rows_per_chunk):
        N += oracle.objective_parts(row_chunk(g, r0, r1), U64, p)[0]
    return N, oracle.p_norm_p(U64, p)


def oracle_delta(g, U64, p, rows_per_chunk=400_000):
    """Delta_p u of every row, block by block."""
    out = np.zeros_like(U64)
    for r0, r1 in chunks(g.n, rows_per_chunk):
        out[r0:r1] = oracle.p_laplacian(row_chunk(g, r0, r1), U64, p)[r0:r1]
    return out


def oracle_grad(g, U64, p, N, D, delta):
    """The Euclidean gradient from Delta_p u and the column sums N, D."""
    return (p / D) * (delta - (N / D) * oracle.phi_p(U64, p))


def star(g, i):
    """(vertices, graph): vertex i first, then its neighbours; only the
    centre's row is stored (its entries in W's order)."""
    nb = g.col[g.rowptr[i]:g.rowptr[i + 1]].astype(np.int64)
    w = g.val[g.rowptr[i]:g.rowptr[i + 1]]
    verts = np.concatenate([[i], nb])
    rp = np.concatenate([[0], np.full(verts.size, nb.size)]).astype(np.int64)
    return verts, wl.CSRGraph(verts.size, rp, np.arange(1, verts.size, dtype=np.int32), w)


def oracle_delta_rows(g, U64, p, rows):
    """Delta_p u on the given rows (star of each row)."""
    out = np.zeros((rows.size, U64.shape[1]))
    for t, i in enumerate(rows):
        verts, s = star(g, i)
        out[t] = oracle.p_laplacian(s, U64[verts], p)[0]
    return out


def oracle_sparse_rows(g, U64, V64, p, rows):
    """(Hess N v)_i = p(p-1) sum_j w_ij |d_ij|^(p-2) (v_i - v_j) on the given
    rows, read off Algorithm 1's form on each row's star: its centre row is
    ((Hess N v)_i - lambda_s (Hess D v)_i) / D_s with the star's own N_s, D_s,
    lambda_s = N_s / D_s."""
    c = p * (p - 1.0)
    out = np.zeros((rows.size, U64.shape[1]))
    for t, i in enumerate(rows):
        verts, s = star(g, i)
        Us, Vs = U64[verts], V64[verts]
        Ns, Ds = oracle.objective_parts(s, Us, p)
        a1 = oracle.alg1_sparse_hvp(s, Us, Vs, p)[0]
        out[t] = Ds * a1 + (Ns / Ds) * c * oracle.abs_pow_pm2(Us[0], p) * Vs[0]
    return out


def oracle_hvp_rows(g, U64, V64, p, rows, N, D, delta):
    """Rows of the exact Hessian product: the sparse part on each row's star,
    the vertex part, and the rank-two terms with the column dots
    <g_N, v> = p <Delta_p u, v> and <g_D, v> = p <phi_p(u), v> taken over
    every row."""
    c = p * (p - 1.0)
    lam = N / D
    cN = p * np.sum(delta * V64, axis=0)
    cD = p * np.sum(oracle.phi_p(U64, p) * V64, axis=0)
    Ur, Vr = U64[rows], V64[rows]
    sparse = oracle_sparse_rows(g, U64, V64, p, rows)
    vertex = c * oracle.abs_pow_pm2(Ur, p) * Vr
    gN = p * delta[rows]
    gD = p * oracle.phi_p(Ur, p)
    return (sparse - lam * vertex) / D - (gN * cD + gD * cN - 2.0 * lam * gD * cD) / D ** 2


def grad_scale_rows(g, U64, p, rows, N, D):
    """|(p/D) Delta_p u| + |(p/D) lambda phi_p(u)| term by term on the given
    rows: the magnitude the gradient's rounding is measured against."""
    out = np.zeros((rows.size, U64.shape[1]))
    for t, i in enumerate(rows):
        nb = g.col[g.rowptr[i]:g.rowptr[i + 1]].astype(np.int64)
        w = g.val[g.rowptr[i]:g.rowptr[i + 1]].astype(np.float64)
        s = (w[:, None] * np.abs(U64[i] - U64[nb]) ** (p - 1.0)).sum(0)
        out[t] = (p / D) * (s + (N / D) * np.abs(U64[i]) ** (p - 1.0))
    return out


def grad_scale(g, U64, p, N, D, rows_per_chunk=400_000):
    """grad_scale_rows for every row, block by block."""
    out = np.zeros_like(U64)
    for r0, r1 in chunks(g.n, rows_per_chunk):
        cg = row_chunk(g, r0, r1)
        rows = np.repeat(np.arange(r0, r1), np.diff(cg.rowptr[r0:r1 + 1]))
        col = cg.col.astype(np.int64)
        w = cg.val.astype(np.float64)
        for l in range(U64.shape[1]):
            t = w * np.abs(U64[rows, l] - U64[col, l]) ** (p - 1.0)
            out[r0:r1, l] = np.bincount(rows - r0, weights=t, minlength=r1 - r0)
    return (p / D) * (out + (N / D) * np.abs(U64) ** (p - 1.0))
