"""k-means discretisation and the RCut metric, in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper discretises the final U with k-means (Section 1) and scores the
clusters with RCut(C_1..C_c) = sum_i cut(C_i, complement C_i) / |C_i|
(Section 3.1).  It gives no k-means details; the reading taken here:

  * Lloyd's algorithm on the rows of U (no row normalisation), as many
    clusters as columns unless told otherwise;
  * k-means++ seeding (Arthur & Vassilvitskii, 2007): the first centre is row
    floor(u n); each further centre is the first row i whose running sum of
    D^2 (squared distance to the nearest chosen centre) exceeds u * sum D^2;
  * the uniforms u come from SplitMix64 (Steele, Lea & Flood, 2014; the
    output function of Vigna's public-domain reference), one stream per call
    seeded with `seed`, consumed in order across restarts, u = (x >> 11) 2^-53;
  * squared distances accumulate dimension by dimension in index order,
    t = x_c - mu_c, acc = acc + t*t, each operation rounded once;
  * assignment ties go to the smallest centre index; an empty cluster is
    re-seeded, in increasing cluster order, at the row farthest from its
    assigned centre (first such row), that row then excluded;
  * stop when an assignment changes no label, or after max_iter updates;
  * several restarts, the one with the smallest inertia kept (first on ties).
RCut: cut(C, complement C) = sum over i in C, j not in C of w_ij; empty
clusters contribute nothing.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15, then the xor-shift-multiply
    output mix (shifts 30, 27, 31; multipliers 0xBF58476D1CE4E5B9,
    0x94D049BB133111EB)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def next_double(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def sq_dist_to(X, c):
    """Squared distance of every row of X to the point c, accumulated in
    dimension order with one rounding per operation."""
    acc = np.zeros(X.shape[0])
    for j in range(X.shape[1]):
        t = X[:, j] - c[j]
        acc = acc + t * t
    return acc


def _all_sq_dist(X, centers):
    return np.stack([sq_dist_to(X, centers[c]) for c in range(centers.shape[0])], axis=1)


def kmeans_pp(X, n_clusters, rng: SplitMix64):
    """k-means++ seeding; returns the (n_clusters x dim) initial centres."""
    n = X.shape[0]
    first = min(int(rng.next_double() * n), n - 1)
    centers = [X[first].copy()]
    d2 = sq_dist_to(X, X[first])
    for _ in range(1, n_clusters):
        u = rng.next_double()
        cum = np.cumsum(d2)
        total = cum[-1]
        if total > 0.0:
            idx = min(int(np.searchsorted(cum, u * total, side="right")), n - 1)
        else:
            idx = min(int(u * n), n - 1)
        centers.append(X[idx].copy())
        d2 = np.minimum(d2, sq_dist_to(X, X[idx]))
    return np.array(centers)


def lloyd(X, centers, max_iter):
    """Lloyd iterations from the given centres; returns (labels, centres,
    inertia, iterations)."""
    C = centers.shape[0]
    centers = centers.copy()
    labels = np.argmin(_all_sq_dist(X, centers), axis=1)
    it = 0
    while it < max_iter:
        it += 1
        dist_own = _all_sq_dist(X, centers)[np.arange(X.shape[0]), labels]
        counts = np.bincount(labels, minlength=C)
        new_centers = np.zeros_like(centers)
        for c in range(C):
            if counts[c] > 0:
                new_centers[c] = X[labels == c].sum(axis=0) / counts[c]
        for c in range(C):
            if counts[c] == 0:
                far = int(np.argmax(dist_own))
                new_centers[c] = X[far]
                dist_own[far] = -1.0
        centers = new_centers
        new_labels = np.argmin(_all_sq_dist(X, centers), axis=1)
        if np.array_equal(new_labels, labels):
            break
        labels = new_labels
    inertia = float(np.sum(_all_sq_dist(X, centers)[np.arange(X.shape[0]), labels]))
    return labels.astype(np.int32), centers, inertia, it


def kmeans(X, n_clusters, seed=0, restarts=10, max_iter=300):
    """k-means++ + Lloyd with restarts; returns (labels, centres, inertia)."""
    X = np.asarray(X, dtype=np.float64)
    rng = SplitMix64(seed)
    best = None
    for _ in range(restarts):
        init = kmeans_pp(X, n_clusters, rng)
        labels, centers, inertia, _ = lloyd(X, init, max_iter)
        if best is None or inertia < best[2]:
            best = (labels, centers, inertia)
    return best


def rcut(g, labels, n_clusters=None):
    """RCut = sum_c cut(C_c, complement)/|C_c| over non-empty clusters (Section 3.1)."""
    labels = np.asarray(labels, dtype=np.int64)
    C = int(labels.max()) + 1 if n_clusters is None else n_clusters
    rowptr = np.asarray(g.rowptr, dtype=np.int64)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rowptr))
    col = np.asarray(g.col, dtype=np.int64)
    w = np.asarray(g.val, dtype=np.float64)
    cross = labels[rows] != labels[col]
    cut = np.bincount(labels[rows][cross], weights=w[cross], minlength=C)
    size = np.bincount(labels, minlength=C)
    nz = size > 0
    return float(np.sum(cut[nz] / size[nz]))
