"""GPU parity of k-means, RCut and the full solve against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_26975_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_26975_gb300 import build
    build.build()
    from paper_2605_26975_gb300 import api as A
    return A


def blobs(seed, n, dim, C, spread=0.15, dtype=np.float32):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1, 1, (C, dim))
    X = centers[rng.integers(0, C, n)] + spread * rng.standard_normal((n, dim))
    return X.astype(dtype)


def same_partition(a, b):
    """True when the two labelings agree up to a permutation of labels."""
    a, b = np.asarray(a), np.asarray(b)
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


@pytest.mark.parametrize("n,dim,C,dtype", [(5000, 4, 4, np.float32), (20000, 8, 8, np.float32),
                                           (3000, 3, 5, np.float64), (257, 16, 16, np.float32)])
def test_kmeans_matches_oracle(api, n, dim, C, dtype):
    X = blobs(n + dim, n, dim, C, dtype=dtype)
    lab, cent, inertia = api.kmeans(torch.from_numpy(X).cuda(), C, seed=7, restarts=4, max_iter=100)
    ref_lab, ref_cent, ref_inertia = oracle.kmeans(X.astype(np.float64), C, seed=7, restarts=4,
                                                   max_iter=100)
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    assert abs(inertia - ref_inertia) <= 1e-10 * ref_inertia
    assert np.allclose(cent.cpu().numpy(), ref_cent, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n,dim,C,dtype", [(4000, 16, 64, np.float32), (64, 1, 64, np.float32),
                                           (3000, 5, 7, np.float32), (2500, 16, 64, np.float64)])
def test_kmeans_extreme_shapes(api, n, dim, C, dtype):
    # the most clusters, as many clusters as rows, a row width off the
    # register buckets (one load per entry), and FP64 rows with 64 clusters
    X = blobs(n * 7 + C, n, dim, C, spread=0.3, dtype=dtype)
    lab, cent, inertia = api.kmeans(torch.from_numpy(X).cuda(), C, seed=11, restarts=2, max_iter=50)
    ref_lab, ref_cent, ref_inertia = oracle.kmeans(X.astype(np.float64), C, seed=11, restarts=2,
                                                   max_iter=50)
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    assert abs(inertia - ref_inertia) <= 1e-10 * max(ref_inertia, 1e-300)
    assert np.allclose(cent.cpu().numpy(), ref_cent, rtol=1e-10, atol=1e-12)


def test_kmeans_empty_cluster_and_duplicates(api):
    # heavy duplicates: k-means++ can only pick distinct rows when D^2 > 0
    X = np.repeat(np.array([[0, 0], [1, 0], [0, 1], [5, 5]], dtype=np.float32), 50, axis=0)
    lab, cent, inertia = api.kmeans(torch.from_numpy(X).cuda(), 4, seed=3, restarts=3)
    ref_lab, _, ref_inertia = oracle.kmeans(X.astype(np.float64), 4, seed=3, restarts=3)
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    assert inertia == ref_inertia == 0.0


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1e3, 1e30])
def test_kmeans_row_magnitudes(api, scale):
    # the member sums of FP32 rows are exact fixed-point sums scaled by
    # 2^q from max |x|: large q, negative q, and rows too small for a finite
    # scale (the FP64 sums) all agree with the oracle
    X = (blobs(3, 4000, 8, 5) * np.float32(scale)).astype(np.float32)
    lab, cent, inertia = api.kmeans(torch.from_numpy(X).cuda(), 5, seed=2, restarts=2, max_iter=60)
    ref_lab, ref_cent, ref_inertia = oracle.kmeans(X.astype(np.float64), 5, seed=2, restarts=2,
                                                   max_iter=60)
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    assert abs(inertia - ref_inertia) <= 1e-10 * ref_inertia
    assert np.allclose(cent.cpu().numpy(), ref_cent, rtol=1e-10, atol=1e-12 * scale)


def test_kmeans_rejects_non_finite_rows(api):
    X = blobs(4, 500, 4, 3)
    X[17, 2] = np.nan
    with pytest.raises(api._abi.PspecError, match="NaN"):
        api.kmeans(torch.from_numpy(X).cuda(), 3)


@pytest.mark.parametrize("max_iter", [0, 1, 3, 8, 9, 17, 300])
def test_kmeans_iteration_cap(api, max_iter):
    # overlapping blobs converge slowly, so most caps stop Lloyd before a
    # fixed point, at every offset inside a chunk of device-side iterations
    X = blobs(11, 6000, 3, 6, spread=0.8)
    lab, cent, inertia = api.kmeans(torch.from_numpy(X).cuda(), 6, seed=5, restarts=2, max_iter=max_iter)
    ref_lab, ref_cent, ref_inertia = oracle.kmeans(X.astype(np.float64), 6, seed=5, restarts=2,
                                                   max_iter=max_iter)
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    assert abs(inertia - ref_inertia) <= 1e-10 * ref_inertia
    assert np.allclose(cent.cpu().numpy(), ref_cent, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("seed,max_iter", [(1, 1), (2, 2), (3, 9), (4, 300)])
def test_kmeans_more_clusters_than_points(api, seed, max_iter):
    # 3 distinct rows, 5 clusters: seeding repeats rows, the repeated centres
    # stay empty and are re-seeded at the farthest rows while no label
    # changes -- Lloyd must still stop at that first unchanged assignment
    X = np.repeat(np.array([[0, 0], [2, 0], [0, 3]], dtype=np.float32), [7, 5, 9], axis=0)
    lab, cent, inertia = api.kmeans(torch.from_numpy(X).cuda(), 5, seed=seed, restarts=2,
                                    max_iter=max_iter)
    ref_lab, ref_cent, ref_inertia = oracle.kmeans(X.astype(np.float64), 5, seed=seed, restarts=2,
                                                   max_iter=max_iter)
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    assert inertia == ref_inertia
    assert np.array_equal(cent.cpu().numpy(), ref_cent)


def test_rcut_matches_oracle(api):
    g = wl.sbm_sampled(np.random.default_rng(2), 5000, 5, 12.0, 0.8)
    G = api.Graph.from_csr(g)
    rng = np.random.default_rng(3)
    for C in (2, 5, 9):
        lab = rng.integers(0, C, g.n).astype(np.int32)
        got = G.rcut(torch.from_numpy(lab).cuda(), C)
        assert abs(got - oracle.rcut(g, lab, C)) <= 1e-12 * got


def test_rcut_rejects_bad_labels(api):
    from paper_2605_26975_gb300 import _abi
    g = wl.sbm_sampled(np.random.default_rng(2), 500, 2, 8.0, 0.8)
    G = api.Graph.from_csr(g)
    lab = np.zeros(g.n, dtype=np.int32)
    lab[7] = 3
    with pytest.raises(_abi.PspecError):
        G.rcut(torch.from_numpy(lab).cuda(), 3)


def test_p2_solve_path_graph_closed_form(api):
    n, k = 40, 3
    a = np.arange(n - 1)
    g = wl.csr_from_undirected(n, a, a + 1, np.ones(n - 1))
    G = api.Graph.from_csr(g)
    U0 = torch.from_numpy(wl.orthonormal_block(5, n, k, np.float64)).cuda()
    U, lab, rc, st, status = G.solve(U0, [2.0], api.default_opts(max_outer=60, gtol_rel=1e-10))
    ref = sum(2 - 2 * math.cos(math.pi * j / n) for j in range(k))
    assert abs(st["f"][0] - ref) <= 1e-9 * ref
    Uc = U.cpu().numpy()
    assert np.allclose(Uc.T @ Uc, np.eye(k), atol=1e-12)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_p2_solve_matches_eigensolver_on_sbm4(api, dtype):
    g = wl.make_graph("sbm4")
    G = api.Graph.from_csr(g)
    U0 = torch.from_numpy(wl.orthonormal_block(2000, g.n, 4, dtype)).cuda()
    U, lab, rc, st, status = G.solve(U0, [2.0], api.default_opts(max_outer=40))
    Wd = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    Wd[rows, g.col] = g.val
    ev = np.linalg.eigvalsh(np.diag(Wd.sum(1)) - Wd)
    tol = 1e-5 if dtype == np.float32 else 1e-10
    assert abs(st["f"][0] - ev[:4].sum()) <= tol * ev[:4].sum()


def test_sbm4_full_solve_matches_oracle(api):
    """The method end to end on the 1,000-vertex SBM: FP32 GPU vs FP64 oracle.
    RCut within 1%, labels equal up to a permutation."""
    g = wl.make_graph("sbm4")
    sched = wl.WORKLOADS["sbm4"]["p_schedule"]
    U0 = wl.orthonormal_block(2000, g.n, 4, np.float32)
    G = api.Graph.from_csr(g)
    U, lab, rc, st, status = G.solve(torch.from_numpy(U0).cuda(), sched, api.default_opts())
    _, ref_lab, ref_rc, stages = oracle.solve(g, U0.astype(np.float64), sched)
    assert abs(rc - ref_rc) <= 0.01 * ref_rc
    assert same_partition(lab.cpu().numpy(), ref_lab)
    # the p = 2 stage reaches the same minimum
    assert abs(st["f"][0] - stages[0]["f"]) <= 1e-5 * stages[0]["f"]


def test_sbm4_plain_fp64_solve_tracks_oracle(api):
    g = wl.make_graph("sbm4")
    sched = (2.0, 1.8, 1.6)
    U0 = wl.orthonormal_block(2000, g.n, 4, np.float64)
    G = api.Graph.from_csr(g)
    U, lab, rc, st, status = G.solve(torch.from_numpy(U0).cuda(), sched, api.default_opts())
    _, ref_lab, ref_rc, stages = oracle.solve(g, U0, sched)
    for s_gpu, s_ref in zip(st["f"], stages):
        assert abs(s_gpu - s_ref["f"]) <= 1e-7 * s_ref["f"]
    assert abs(rc - ref_rc) <= 1e-12 * ref_rc
    assert same_partition(lab.cpu().numpy(), ref_lab)


def test_solve_rejects_bad_schedule(api):
    from paper_2605_26975_gb300 import _abi
    g = wl.make_graph("sbm4")
    G = api.Graph.from_csr(g)
    U0 = torch.from_numpy(wl.orthonormal_block(1, g.n, 4, np.float32)).cuda()
    for sched in ([1.5, 1.8], [2.2], [1.0]):
        with pytest.raises(_abi.PspecError):
            G.solve(U0, sched)


def test_graph_replayed_solve_equals_eager_solve(api):
    """The solve replays chunks of tCG iterations as CUDA graphs; with kernel
    timing on it launches every kernel eagerly.  Both run the same kernels in
    the same order, so the results are bit-identical."""
    g = wl.make_graph("sbm4")
    sched = (2.0, 1.6)
    U0 = torch.from_numpy(wl.orthonormal_block(2000, g.n, 4, np.float32)).cuda()
    G = api.Graph.from_csr(g)
    U1, lab1, rc1, st1, _ = G.solve(U0, sched, api.default_opts())
    G.set_timing(True)
    U2, lab2, rc2, st2, _ = G.solve(U0, sched, api.default_opts())
    G.set_timing(False)
    assert torch.equal(U1, U2) and torch.equal(lab1, lab2)
    assert rc1 == rc2 and st1["hvp_calls"] == st2["hvp_calls"]
