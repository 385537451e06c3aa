"""Pins of the oracle's k-means and RCut (SplitMix64 against its published
reference outputs; k-means against brute-force optimal partitions and the
Lloyd fixed point; RCut against dense double loops and a closed form)."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2605_26975_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_graph(Wd):
    n = Wd.shape[0]
    iu, ju = np.nonzero(np.triu(Wd, 1))
    return wl.csr_from_undirected(n, iu, ju, Wd[iu, ju], np.float64)


def test_splitmix64_reference_outputs():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for row in rows:
        rng = oracle.SplitMix64(int(row[0]))
        assert [rng.next_u64() for _ in row[1:]] == [int(x) for x in row[1:]]
    u = oracle.SplitMix64(7)
    vals = [u.next_double() for _ in range(1000)]
    assert min(vals) >= 0.0 and max(vals) < 1.0


def _inertia(X, labels, C):
    tot = 0.0
    for c in range(C):
        pts = X[labels == c]
        if len(pts):
            tot += ((pts - pts.mean(axis=0)) ** 2).sum()
    return tot


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_kmeans_matches_brute_force_optimum(seed):
    rng = np.random.default_rng(seed)
    C, n = 3, 9
    centers = rng.uniform(-5, 5, (C, 2))
    X = centers[np.arange(n) % C] + 0.3 * rng.standard_normal((n, 2))
    best = min(_inertia(X, np.array(lab), C)
               for lab in itertools.product(range(C), repeat=n) if len(set(lab)) == C)
    labels, cent, inertia = oracle.kmeans(X, C, seed=seed)
    assert abs(inertia - best) <= 1e-12 * max(1.0, best)


def test_kmeans_fixed_point():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((300, 3))
    labels, cent, inertia = oracle.kmeans(X, 5, seed=11)
    d = np.stack([((X - c) ** 2).sum(1) for c in cent], axis=1)
    assert np.array_equal(labels, d.argmin(axis=1))
    for c in range(5):
        assert np.allclose(cent[c], X[labels == c].mean(axis=0), atol=1e-13)
    assert abs(inertia - _inertia(X, labels, 5)) <= 1e-10 * inertia


def test_kmeans_empty_cluster_reseed():
    # four points, two of them duplicated: a centre can lose all its points
    X = np.array([[0.0, 0.0], [0.0, 0.0], [10.0, 0.0], [10.0, 0.0], [5.0, 9.0]])
    centers = np.array([[0.0, 0.0], [10.0, 0.0], [100.0, 100.0]])
    labels, cent, inertia, it = oracle.lloyd(X, centers, 10)
    assert len(set(labels.tolist())) == 3 and inertia == 0.0


def test_rcut_brute_force():
    rng = np.random.default_rng(6)
    n, C = 11, 3
    A = np.triu((rng.random((n, n)) < 0.5) * rng.uniform(0.1, 2.0, (n, n)), 1)
    Wd = A + A.T
    g = dense_graph(Wd)
    labels = rng.integers(0, C, n)
    ref = 0.0
    for c in range(C):
        members = [i for i in range(n) if labels[i] == c]
        if members:
            cut = sum(Wd[i, j] for i in members for j in range(n) if labels[j] != c)
            ref += cut / len(members)
    assert abs(oracle.rcut(g, labels, C) - ref) <= 1e-13 * ref


def test_rcut_two_cliques():
    m = 6
    n = 2 * m
    Wd = np.zeros((n, n))
    Wd[:m, :m] = 1
    Wd[m:, m:] = 1
    np.fill_diagonal(Wd, 0)
    Wd[m - 1, m] = Wd[m, m - 1] = 1
    g = dense_graph(Wd)
    labels = np.repeat([0, 1], m)
    assert oracle.rcut(g, labels) == 2.0 / m
