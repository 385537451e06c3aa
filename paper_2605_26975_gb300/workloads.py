"""Seeded synthetic inputs for p-spectral clustering: graphs and initial blocks.

This module is the one place both the CUDA path (through its tests and the
benchmark) and the FP64 CPU oracle take their inputs from.  It holds none of
the method's arithmetic: it only draws graphs and dense blocks from numpy's
PCG64 generator and packs symmetric weight matrices as CSR.

The paper measures on SuiteSparse Delaunay graphs (n = 2^r, about 6n stored
entries, Section 3).  Those matrices are not available here, so the graphs
below are synthetic stand-ins with the sizes, degree distributions and weight
distributions of the five workload shapes this library is tested and
benchmarked on:

  sbm4        stochastic block model, n=1,000, 4 equal blocks, Bernoulli
              0.05 inside a block and 0.002 across, unit weights (k=4)
  knn_gmm     200,000 points from 8 isotropic 2-D Gaussians (means uniform
              in [0,10]^2, sigma 0.5), 10 nearest neighbours symmetrised by
              union, w = exp(-d^2/0.25)  (k=8)
  grid3d      200^3 6-neighbour grid, w ~ U[0.5,1.5], 0.1% of the edges
              replaced by random long-range links (k=8)
  dcsbm       degree-corrected SBM, n=1,000,000, 16 blocks, Pareto degree
              propensities with tail exponent 2.5, mean degree 16,
              w ~ U[0.1,1]  (k=16)
  sbm_batch   512 SBMs with n log-uniform in [500, 50,000], 2..8 blocks,
              mean degree 8..20, unit weights, k in {2,4,8} per graph
  delaunayR   Delaunay triangulation of 2^R points uniform in the unit
              square, unit weights (about 6n stored entries), R = 16..19:
              the construction of the paper's Delaunay matrices, drawn
              afresh  (k=4)

Every graph is undirected: both triangles are stored, rows hold sorted column
indices, there are no self loops and no duplicate entries.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class CSRGraph:
    """A symmetric, non-negative weight matrix W in CSR form (both triangles)."""

    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray     # int32[nnz]
    val: np.ndarray     # float32 or float64[nnz]
    labels: np.ndarray | None = None  # planted block of each vertex, if any

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def astype(self, dtype) -> "CSRGraph":
        return CSRGraph(self.n, self.rowptr, self.col, self.val.astype(dtype), self.labels)


def csr_from_undirected(n: int, a: np.ndarray, b: np.ndarray, w: np.ndarray,
                        val_dtype=np.float32) -> CSRGraph:
    """Pack undirected edges {a_e, b_e} with weight w_e into a symmetric CSR.

    Self loops are dropped; a pair given twice keeps its first weight.
    """
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    keep = a != b
    a, b, w = a[keep], b[keep], w[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = lo * n + hi
    key, first = np.unique(key, return_index=True)
    lo, hi, w = key // n, key % n, w[first]
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    ww = np.concatenate([w, w])
    order = np.argsort(rows * n + cols, kind="stable")
    rows, cols, ww = rows[order], cols[order], ww[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSRGraph(n, rowptr, cols.astype(np.int32), ww.astype(val_dtype))


# --------------------------------------------------------------------------
# graphs
# --------------------------------------------------------------------------

def sbm_bernoulli(seed: int, n: int = 1000, blocks: int = 4, p_in: float = 0.05,
                  p_out: float = 0.002, val_dtype=np.float32) -> CSRGraph:
    """SBM drawn pair by pair: each upper-triangle pair is an edge with
    probability p_in (same block) or p_out (different blocks); unit weights.
    Blocks are contiguous and equal (vertex i is in block i*blocks//n)."""
    rng = np.random.default_rng(seed)
    label = (np.arange(n) * blocks) // n
    iu, ju = np.triu_indices(n, k=1)
    prob = np.where(label[iu] == label[ju], p_in, p_out)
    hit = rng.random(iu.size) < prob
    g = csr_from_undirected(n, iu[hit], ju[hit], np.ones(int(hit.sum())), val_dtype)
    g.labels = label.astype(np.int32)
    return g


def knn_gaussian_mixture(seed: int, n: int = 200_000, mixtures: int = 8, sigma: float = 0.5,
                         neighbours: int = 10, box: float = 10.0, bandwidth: float = 0.25,
                         val_dtype=np.float32) -> CSRGraph:
    """kNN similarity graph of points from a mixture of isotropic 2-D Gaussians.

    Means are uniform in [0, box]^2; each component holds n/mixtures points;
    the point order is shuffled.  Each point is joined to its `neighbours`
    nearest other points (exact, kd-tree), the relation is symmetrised by
    union and w_ij = exp(-|x_i - x_j|^2 / bandwidth), rounded to float32.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    means = rng.uniform(0.0, box, size=(mixtures, 2))
    comp = np.repeat(np.arange(mixtures), n // mixtures)
    comp = np.concatenate([comp, np.arange(n - comp.size) % mixtures])
    pts = means[comp] + sigma * rng.standard_normal((n, 2))
    perm = rng.permutation(n)
    pts, comp = pts[perm], comp[perm]
    tree = cKDTree(pts)
    dist, idx = tree.query(pts, k=neighbours + 1)
    a = np.repeat(np.arange(n), neighbours)
    b = idx[:, 1:].reshape(-1)
    d = dist[:, 1:].reshape(-1)
    w = np.exp(-(d * d) / bandwidth).astype(np.float32).astype(np.float64)
    g = csr_from_undirected(n, a, b, w, val_dtype)
    g.labels = comp.astype(np.int32)
    return g


def grid3d_longrange(seed: int, side: int = 200, frac_long: float = 1e-3, w_lo: float = 0.5,
                     w_hi: float = 1.5, val_dtype=np.float32) -> CSRGraph:
    """side^3 grid with 6-neighbour edges (x fastest), w ~ U[w_lo, w_hi].

    A fraction `frac_long` of the undirected edges, chosen uniformly, is
    deleted and replaced by as many uniformly random vertex pairs that are
    neither self loops, grid-adjacent candidates, nor repeated.
    """
    rng = np.random.default_rng(seed)
    n = side ** 3
    idx = np.arange(n, dtype=np.int64)
    x = idx % side
    y = (idx // side) % side
    z = idx // (side * side)
    parts_a, parts_b = [], []
    for coord, step in ((x, 1), (y, side), (z, side * side)):
        src = idx[coord < side - 1]
        parts_a.append(src)
        parts_b.append(src + step)
    del x, y, z, idx
    a = np.concatenate(parts_a)
    b = np.concatenate(parts_b)
    del parts_a, parts_b
    m = a.size
    w = rng.uniform(w_lo, w_hi, size=m)
    n_long = int(round(frac_long * m))
    drop = rng.choice(m, size=n_long, replace=False)
    keep = np.ones(m, dtype=bool)
    keep[drop] = False
    a, b, w = a[keep], b[keep], w[keep]
    # long-range links: reject self loops and any pair whose index gap is a
    # grid step (a superset of the grid edges), then de-duplicate
    new_a, new_b = [], []
    have = 0
    seen = set()
    while have < n_long:
        ca = rng.integers(0, n, size=2 * (n_long - have) + 16)
        cb = rng.integers(0, n, size=ca.size)
        gap = np.abs(ca - cb)
        ok = (gap != 0) & (gap != 1) & (gap != side) & (gap != side * side)
        for i, j in zip(ca[ok].tolist(), cb[ok].tolist()):
            key = (min(i, j), max(i, j))
            if key in seen:
                continue
            seen.add(key)
            new_a.append(i)
            new_b.append(j)
            have += 1
            if have == n_long:
                break
    a = np.concatenate([a, np.asarray(new_a, dtype=np.int64)])
    b = np.concatenate([b, np.asarray(new_b, dtype=np.int64)])
    w = np.concatenate([w, rng.uniform(w_lo, w_hi, size=n_long)])
    return csr_from_undirected(n, a, b, w, val_dtype)


def dcsbm_powerlaw(seed: int, n: int = 1_000_000, blocks: int = 16, mean_degree: float = 16.0,
                   tail: float = 2.5, intra: float = 0.8, w_lo: float = 0.1, w_hi: float = 1.0,
                   val_dtype=np.float32) -> CSRGraph:
    """Degree-corrected SBM with Chung-Lu style edge sampling.

    Propensities theta_i follow a Pareto law with density proportional to
    theta^-tail on [1, inf).  Vertices fall into `blocks` equal blocks in a
    random order.  About n*mean_degree/2 undirected edges are drawn: a
    fraction `intra` inside blocks (block chosen with weight S_a^2, S_a the
    block's propensity mass), the rest across block pairs (weight S_a*S_b);
    endpoints are drawn within a block with probability proportional to
    theta.  Repeats and self loops are removed; w ~ U[w_lo, w_hi].
    """
    rng = np.random.default_rng(seed)
    theta = 1.0 + rng.pareto(tail - 1.0, size=n)
    block = np.empty(n, dtype=np.int64)
    block[rng.permutation(n)] = (np.arange(n) * blocks) // n
    members = [np.flatnonzero(block == a) for a in range(blocks)]
    cums = [np.cumsum(theta[mb]) for mb in members]
    mass = np.array([c[-1] for c in cums])
    m_total = int(round(n * mean_degree / 2))

    def draw(a, count):
        u = rng.uniform(0.0, mass[a], size=count)
        pos = np.minimum(np.searchsorted(cums[a], u, side="right"), members[a].size - 1)
        return members[a][pos]

    ea, eb = [], []
    m_in = int(round(intra * m_total))
    w_in = mass ** 2 / np.sum(mass ** 2)
    cnt_in = rng.multinomial(m_in, w_in)
    for a in range(blocks):
        ea.append(draw(a, cnt_in[a]))
        eb.append(draw(a, cnt_in[a]))
    pairs = [(a, b) for a in range(blocks) for b in range(a + 1, blocks)]
    w_out = np.array([mass[a] * mass[b] for a, b in pairs])
    cnt_out = rng.multinomial(m_total - m_in, w_out / w_out.sum())
    for (a, b), c in zip(pairs, cnt_out):
        ea.append(draw(a, c))
        eb.append(draw(b, c))
    a = np.concatenate(ea)
    b = np.concatenate(eb)
    w = rng.uniform(w_lo, w_hi, size=a.size)
    g = csr_from_undirected(n, a, b, w, val_dtype)
    g.labels = block.astype(np.int32)
    return g


def sbm_sampled(rng: np.random.Generator, n: int, blocks: int, mean_degree: float,
                intra: float, val_dtype=np.float32) -> CSRGraph:
    """SBM with about n*mean_degree/2 uniformly sampled edges, a fraction
    `intra` inside equal contiguous blocks; unit weights."""
    label = (np.arange(n) * blocks) // n
    starts = np.searchsorted(label, np.arange(blocks))
    sizes = np.bincount(label, minlength=blocks)
    m = int(round(n * mean_degree / 2))
    m_in = int(round(intra * m))
    ba = rng.integers(0, blocks, size=m_in)
    a_in = starts[ba] + (rng.random(m_in) * sizes[ba]).astype(np.int64)
    b_in = starts[ba] + (rng.random(m_in) * sizes[ba]).astype(np.int64)
    m_out = m - m_in
    b1 = rng.integers(0, blocks, size=m_out)
    b2 = (b1 + rng.integers(1, blocks, size=m_out)) % blocks
    a_out = starts[b1] + (rng.random(m_out) * sizes[b1]).astype(np.int64)
    b_out = starts[b2] + (rng.random(m_out) * sizes[b2]).astype(np.int64)
    a = np.concatenate([a_in, a_out])
    b = np.concatenate([b_in, b_out])
    g = csr_from_undirected(n, a, b, np.ones(a.size), val_dtype)
    g.labels = label.astype(np.int32)
    return g


@dataclasses.dataclass
class GraphBatch:
    """Many graphs concatenated: graph g owns vertices node_off[g]..node_off[g+1]
    and its rows of the shared CSR; column indices are global."""

    graphs: list
    node_off: np.ndarray   # int64[G+1]
    k: np.ndarray          # int32[G] columns per graph
    csr: CSRGraph          # the block-diagonal concatenation


def concat_graphs(graphs: list, ks) -> GraphBatch:
    node_off = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum([g.n for g in graphs], out=node_off[1:])
    rowptrs, cols, vals = [np.zeros(1, dtype=np.int64)], [], []
    base = 0
    for g, off in zip(graphs, node_off[:-1]):
        rowptrs.append(g.rowptr[1:] + base)
        cols.append(g.col.astype(np.int64) + off)
        vals.append(g.val)
        base += g.nnz
    n = int(node_off[-1])
    csr = CSRGraph(n, np.concatenate(rowptrs), np.concatenate(cols).astype(np.int32),
                   np.concatenate(vals))
    return GraphBatch(graphs, node_off, np.asarray(ks, dtype=np.int32), csr)


def sbm_batch(seed: int, n_graphs: int = 512, n_lo: int = 500, n_hi: int = 50_000,
              val_dtype=np.float32) -> GraphBatch:
    """Batch of SBMs: n log-uniform in [n_lo, n_hi], 2..8 blocks, mean degree
    U[8,20], 90% of edges inside blocks, unit weights, k in {2,4,8}."""
    rng = np.random.default_rng(seed)
    graphs, ks = [], []
    for _ in range(n_graphs):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        blocks = int(rng.integers(2, 9))
        deg = float(rng.uniform(8.0, 20.0))
        graphs.append(sbm_sampled(rng, n, blocks, deg, 0.9, val_dtype))
        ks.append(int(rng.choice([2, 4, 8])))
    return concat_graphs(graphs, ks)


def delaunay_unit_square(seed: int, n: int, val_dtype=np.float32) -> CSRGraph:
    """Delaunay triangulation of n points drawn uniformly in [0,1]^2 (scipy's
    Qhull), every triangle side an undirected edge of weight 1."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    tri = Delaunay(pts).simplices.astype(np.int64)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [0, 2]]])
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    return csr_from_undirected(n, e[:, 0], e[:, 1], np.ones(len(e)), val_dtype)


# --------------------------------------------------------------------------
# dense blocks
# --------------------------------------------------------------------------

def orthonormal_block(seed: int, n: int, k: int, dtype=np.float32) -> np.ndarray:
    """n x k row-major block: i.i.d. N(0,1) entries, then the Q factor of a
    thin QR with a non-negative diagonal of R, then rounded to `dtype`."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, k))
    q, r = np.linalg.qr(g)
    q = q * np.where(np.diag(r) < 0, -1.0, 1.0)
    return np.ascontiguousarray(q.astype(dtype))


def gaussian_block(seed: int, n: int, k: int, scale: float = 1.0, dtype=np.float32) -> np.ndarray:
    """n x k row-major block of i.i.d. N(0, scale^2) entries, rounded to dtype."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray((scale * rng.standard_normal((n, k))).astype(dtype))


# --------------------------------------------------------------------------
# named workloads (graph seed 1000 + index, block seeds 2000/3000 + index)
# --------------------------------------------------------------------------

WORKLOADS = {
    "sbm4": dict(index=0, k=4, p_schedule=(2.0, 1.8, 1.6, 1.4, 1.2)),
    "knn_gmm": dict(index=1, k=8, p_schedule=tuple(round(2.0 - 0.1 * i, 1) for i in range(10))),
    "grid3d": dict(index=2, k=8, p_schedule=(2.0, 1.6, 1.3, 1.1)),
    "dcsbm": dict(index=3, k=16, p_schedule=(1.3,)),
    "sbm_batch": dict(index=4, k=None, p_schedule=tuple(round(2.0 - 0.1 * i, 1) for i in range(9))),
}
for _r in (16, 17, 18, 19):
    WORKLOADS[f"delaunay{_r}"] = dict(index=5 + _r - 16, k=4,
                                      p_schedule=tuple(round(2.0 - 0.1 * i, 1) for i in range(10)))


def make_graph(name: str, val_dtype=np.float32):
    """Build the named workload's graph (a GraphBatch for sbm_batch)."""
    idx = WORKLOADS[name]["index"]
    seed = 1000 + idx
    if name == "sbm4":
        return sbm_bernoulli(seed, val_dtype=val_dtype)
    if name == "knn_gmm":
        return knn_gaussian_mixture(seed, val_dtype=val_dtype)
    if name == "grid3d":
        return grid3d_longrange(seed, val_dtype=val_dtype)
    if name == "dcsbm":
        return dcsbm_powerlaw(seed, val_dtype=val_dtype)
    if name == "sbm_batch":
        return sbm_batch(seed, val_dtype=val_dtype)
    if name.startswith("delaunay"):
        return delaunay_unit_square(seed, 1 << int(name[len("delaunay"):]), val_dtype=val_dtype)
    raise KeyError(name)


def make_blocks(name: str, n: int, k: int, dtype=np.float32):
    """(U, V) for per-call timing and parity: U orthonormal (seed 2000+i),
    V i.i.d. N(0,1) (seed 3000+i)."""
    idx = WORKLOADS[name]["index"]
    return (orthonormal_block(2000 + idx, n, k, dtype),
            gaussian_block(3000 + idx, n, k, dtype=dtype))
