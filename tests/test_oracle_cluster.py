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


def test_kmeans_pp_hand_example():
    """k-means++ seeding on the five points 0, 1, 3, 7, 15 with SplitMix64(0),
    worked by hand from the golden outputs of that stream:
      u0 = 16294208416658607535 / 2^64 = 0.88331...  -> first centre row
           floor(5 u0) = 4 (x = 15); D^2 = 225, 196, 144, 64, 0 (sum 629)
      u1 = 7960286522194355700 / 2^64 = 0.43153...   -> u1 * 629 = 271.43, first
           running sum of D^2 above it is 421 at row 1 (x = 1);
           D^2 = min(previous, distance to 1) = 1, 0, 4, 36, 0 (sum 41)
      u2 = 487617019471545679 / 2^64 = 0.02643...    -> u2 * 41 = 1.084, first
           running sum above it is 5 at row 2 (x = 3).
    Weighting by D instead of D^2 picks row 0 third; not lowering D^2 to the
    nearest chosen centre picks row 3."""
    X = np.array([[0.0], [1.0], [3.0], [7.0], [15.0]])
    centres = oracle.kmeans_pp(X, 3, oracle.SplitMix64(0))
    assert centres[:, 0].tolist() == [15.0, 1.0, 3.0]


def test_kmeans_pp_draw_follows_d_squared():
    """Over many seeds the second centre, given the first, is drawn with
    probability D^2 / sum D^2 (chi-square goodness of fit, 20,000 draws)."""
    from scipy import stats
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0], [3.0, 1.0], [-2.0, -1.0]])
    n = X.shape[0]
    counts = np.zeros((n, n))
    for seed in range(20_000):
        c = oracle.kmeans_pp(X, 2, oracle.SplitMix64(seed))
        f = int(np.flatnonzero((X == c[0]).all(1))[0])
        s = int(np.flatnonzero((X == c[1]).all(1))[0])
        counts[f, s] += 1
    chi2, dof = 0.0, 0
    for f in range(n):
        d2 = ((X - X[f]) ** 2).sum(1)
        expected = counts[f].sum() * d2 / d2.sum()
        assert counts[f, f] == 0  # a chosen point has D^2 = 0
        m = expected > 0
        chi2 += float((((counts[f] - expected) ** 2)[m] / expected[m]).sum())
        dof += int(m.sum()) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-3, (chi2, dof)
    # the first centre is uniform over the rows
    first = counts.sum(1)
    assert stats.chisquare(first).pvalue > 1e-3


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
