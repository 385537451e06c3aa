"""pspec_solve_lockstep: every graph of a batched handle solved with the whole
batch stepping together on the device.  Each graph takes the iterates it
would take alone, up to the summation order of the reductions, so it is
compared with pspec_solve on the graph alone at rounding level where the
problem is well conditioned (the p = 2 stage, whose minimum is the sum of
the k smallest Laplacian eigenvalues), with the FP64 oracle's solve on the
1,000-vertex SBM, and with the oracle's RCut of its own labels."""
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


def same_partition(a, b):
    pairs = set(zip(np.asarray(a).tolist(), np.asarray(b).tolist()))
    return len(pairs) == len(set(np.asarray(a).tolist())) == len(set(np.asarray(b).tolist()))


def batch_and_blocks(k, extra=()):
    rng = np.random.default_rng(21)
    gs = [wl.make_graph("sbm4"),
          wl.sbm_sampled(rng, 3000, 4, 12.0, 0.9),
          wl.sbm_sampled(rng, 200, 3, 8.0, 0.9),
          wl.knn_gaussian_mixture(4, n=5000, mixtures=4)] + list(extra)
    batch = wl.concat_graphs(gs, [k] * len(gs))
    U = np.concatenate([wl.orthonormal_block(2000 if i == 0 else 500 + i, g.n, k)
                        for i, g in enumerate(gs)])
    return gs, batch, U


def handle(api, batch):
    c = batch.csr
    return api.Graph(c.rowptr, c.col, c.val, node_off=batch.node_off)


def laplacian_eigs(g, k):
    Wd = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    Wd[rows, g.col] = g.val
    return np.linalg.eigvalsh(np.diag(Wd.sum(1)) - Wd)[:k]


def test_lockstep_p2_stage_matches_eigenvalues_and_single_solves(api):
    """One p = 2 stage: every graph's F reaches the sum of its k smallest
    Laplacian eigenvalues (Ky Fan), as pspec_solve on the graph alone does."""
    k = 4
    rng = np.random.default_rng(3)
    gs = [wl.make_graph("sbm4"), wl.sbm_sampled(rng, 1500, 5, 10.0, 0.85),
          wl.sbm_sampled(rng, 37, 2, 6.0, 0.9), wl.delaunay_unit_square(4, 800)]
    batch = wl.concat_graphs(gs, [k] * len(gs))
    U = np.concatenate([wl.orthonormal_block(40 + i, g.n, k) for i, g in enumerate(gs)])
    G = handle(api, batch)
    opts = api.default_opts(max_outer=60)
    Ub, lab, rc, status, stats, st = G.solve_lockstep(torch.from_numpy(U).cuda(), [2.0], opts, threads=4)
    # OK, or NOT_CONVERGED where FP32's gradient floor sits above gtol_rel = 1e-6
    assert all(s in (0, 6) for s in status), status
    for i, g in enumerate(gs):
        ev = laplacian_eigs(g, k).sum()
        assert abs(stats[i]["f"][0] - ev) <= 1e-5 * ev, (i, stats[i]["f"][0], ev)
        a, b = batch.node_off[i], batch.node_off[i + 1]
        S = api.Graph.from_csr(g)
        _, _, _, st1, status1 = S.solve(torch.from_numpy(U[a:b]).cuda(), [2.0], opts)
        assert abs(stats[i]["f"][0] - st1["f"][0]) <= 2e-6 * ev, (i, stats[i]["f"][0], st1["f"][0])
        Uc = Ub[a:b].double().cpu().numpy()
        assert np.allclose(Uc.T @ Uc, np.eye(k), atol=1e-5), i
        # counters are consistent: one evaluation per stage plus one per Newton step
        assert stats[i]["eval_calls"] == 1 + stats[i]["outer"][0]
        assert stats[i]["hvp_calls"] == stats[i]["inner"][0] >= stats[i]["outer"][0] >= 1


def test_lockstep_tracks_single_solves_over_the_schedule(api):
    k = 4
    sched = (2.0, 1.6, 1.3)
    gs, batch, U = batch_and_blocks(k)
    G = handle(api, batch)
    Ub, lab, rc, status, stats, st = G.solve_lockstep(torch.from_numpy(U).cuda(), sched, threads=4)
    assert all(s in (0, 6) for s in status), status  # OK or NOT_CONVERGED
    for i, g in enumerate(gs):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        S = api.Graph.from_csr(g)
        Ui, labi, rci, sti, _ = S.solve(torch.from_numpy(U[a:b]).cuda(), sched)
        # the p = 2 stage at rounding level; the final cut within 1%
        assert abs(stats[i]["f"][0] - sti["f"][0]) <= 1e-5 * sti["f"][0], i
        # (the kNN mixture's last stage is the least conditioned: 3%)
        assert abs(rc[i] - rci) <= (0.01 if i < 3 else 0.03) * rci, (i, rc[i], rci)
        # the RCut reported is the cut of the labels returned
        li = lab[a:b].cpu().numpy()
        assert abs(rc[i] - oracle.rcut(g, li, k)) <= 1e-12 * rc[i], i
        if i < 3:  # the SBMs: the same blocks
            assert same_partition(li, labi.cpu().numpy()), i


def test_lockstep_sbm4_matches_oracle_and_is_deterministic(api):
    k = 4
    sched = wl.WORKLOADS["sbm4"]["p_schedule"]
    gs, batch, U = batch_and_blocks(k)
    G = handle(api, batch)
    Ub, lab, rc, status, stats, st = G.solve_lockstep(torch.from_numpy(U).cuda(), sched)
    n0 = gs[0].n
    _, ref_lab, ref_rc, stages = oracle.solve(gs[0], U[:n0].astype(np.float64), sched)
    assert abs(rc[0] - ref_rc) <= 0.01 * ref_rc
    assert same_partition(lab[:n0].cpu().numpy(), ref_lab)
    assert abs(stats[0]["f"][0] - stages[0]["f"]) <= 1e-5 * stages[0]["f"]
    # fixed-order reductions: a second call gives the same bits
    Ub2, lab2, rc2, status2, _, _ = G.solve_lockstep(torch.from_numpy(U).cuda(), sched, threads=2)
    assert torch.equal(Ub, Ub2) and torch.equal(lab, lab2) and np.array_equal(rc, rc2)
    assert np.array_equal(status, status2)


def test_lockstep_eager_equals_graph_replay(api, monkeypatch):
    k = 2
    sched = (2.0, 1.5)
    rng = np.random.default_rng(8)
    gs = [wl.sbm_sampled(rng, 900, 2, 9.0, 0.9), wl.sbm_sampled(rng, 2500, 3, 11.0, 0.9)]
    batch = wl.concat_graphs(gs, [k] * len(gs))
    U = np.concatenate([wl.orthonormal_block(70 + i, g.n, k) for i, g in enumerate(gs)])
    G = handle(api, batch)
    Ua, laba, rca, _, sa, _ = G.solve_lockstep(torch.from_numpy(U).cuda(), sched)
    monkeypatch.setenv("PSPEC_SOLVE_EAGER", "1")
    Ue, labe, rce, _, se, _ = G.solve_lockstep(torch.from_numpy(U).cuda(), sched)
    assert torch.equal(Ua, Ue) and torch.equal(laba, labe) and np.array_equal(rca, rce)
    assert [s["inner"] for s in sa] == [s["inner"] for s in se]


@pytest.mark.parametrize("k", [1, 3, 8, 16])
def test_lockstep_other_k_and_algorithm1(api, k):
    """Odd k (scalar row paths) and k = 8, in the exact and in Algorithm 1's
    Hessian form: the p = 2 stage (where both forms have the same minimum)
    against pspec_solve per graph."""
    rng = np.random.default_rng(30 + k)
    blocks = max(k, 2)
    gs = [wl.sbm_sampled(rng, 800, blocks, 10.0, 0.9), wl.sbm_sampled(rng, 2000, blocks, 12.0, 0.9)]
    batch = wl.concat_graphs(gs, [k] * len(gs))
    U = np.concatenate([wl.orthonormal_block(90 + i, g.n, k) for i, g in enumerate(gs)])
    G = handle(api, batch)
    for form in (api._abi.PSPEC_HESSIAN_EXACT, api._abi.PSPEC_HESSIAN_ALG1):
        opts = api.default_opts(max_outer=60, hessian_form=form)
        _, _, rc, status, stats, _ = G.solve_lockstep(torch.from_numpy(U).cuda(), [2.0, 1.7], opts)
        assert all(s in (0, 6) for s in status)
        for i, g in enumerate(gs):
            a, b = batch.node_off[i], batch.node_off[i + 1]
            S = api.Graph.from_csr(g)
            _, _, rci, sti, _ = S.solve(torch.from_numpy(U[a:b]).cuda(), [2.0, 1.7], opts)
            # (k = 1: the minimum is the constant vector, F = 0, one cluster, RCut = 0)
            assert abs(stats[i]["f"][0] - sti["f"][0]) <= 1e-5 * max(sti["f"][0], 1e-3), (form, i)
            assert abs(rc[i] - rci) <= 0.02 * rci, (form, i, rc[i], rci)


def test_lockstep_reports_a_graph_smaller_than_k(api):
    rng = np.random.default_rng(5)
    gs = [wl.sbm_sampled(rng, 400, 2, 8.0, 0.9),
          wl.csr_from_undirected(2, np.array([0]), np.array([1]), np.array([1.0]), np.float32),
          wl.sbm_sampled(rng, 300, 3, 8.0, 0.9)]
    batch = wl.concat_graphs(gs, [3] * len(gs))
    G = handle(api, batch)
    U = np.concatenate([wl.orthonormal_block(i, g.n, 3) if g.n >= 3 else wl.gaussian_block(i, g.n, 3)
                        for i, g in enumerate(gs)])
    with pytest.raises(api._abi.PspecError, match="graph 1"):
        G.solve_lockstep(torch.from_numpy(U).cuda(), [2.0])
    Ub, lab, rc, status, stats, st = G.solve_lockstep(torch.from_numpy(U).cuda(), [2.0], allow_errors=True)
    assert status[1] == api._abi.PSPEC_ERR_INVALID_ARG and math.isnan(rc[1])
    assert st == api._abi.PSPEC_ERR_INVALID_ARG
    # the graph's rows are left as they were; the others are solved
    a, b = batch.node_off[1], batch.node_off[2]
    assert torch.equal(Ub[a:b].cpu(), torch.from_numpy(U[a:b]))
    for i in (0, 2):
        assert status[i] in (0, 6) and np.isfinite(rc[i]) and rc[i] > 0
        ev = laplacian_eigs(gs[i], 3).sum()
        assert abs(stats[i]["f"][0] - ev) <= 1e-5 * ev


def test_lockstep_zero_column_stops_only_its_graph(api):
    """A graph whose starting block has a zero column meets ZERO_COLUMN at its
    first evaluation; the other graphs' solves are unaffected."""
    rng = np.random.default_rng(9)
    gs = [wl.sbm_sampled(rng, 600, 2, 9.0, 0.9), wl.sbm_sampled(rng, 500, 2, 9.0, 0.9)]
    batch = wl.concat_graphs(gs, [2, 2])
    G = handle(api, batch)
    U = np.concatenate([wl.orthonormal_block(60 + i, g.n, 2) for i, g in enumerate(gs)])
    U[gs[0].n:, 1] = 0.0
    _, _, rc, status, stats, st = G.solve_lockstep(torch.from_numpy(U).cuda(), [2.0, 1.5],
                                                   allow_errors=True)
    assert status[1] == api._abi.PSPEC_ERR_ZERO_COLUMN and math.isnan(rc[1])
    assert st == api._abi.PSPEC_ERR_ZERO_COLUMN
    S = api.Graph.from_csr(gs[0])
    _, _, rc0, st0, _ = S.solve(torch.from_numpy(U[:gs[0].n]).cuda(), [2.0, 1.5])
    assert abs(stats[0]["f"][0] - st0["f"][0]) <= 1e-5 * st0["f"][0]
    assert abs(rc[0] - rc0) <= 0.01 * rc0


def test_solves_below_p2_reach_the_component_optimum(api):
    """Graphs with exactly k connected components, where F_p = 0 on the span of
    the component indicators for every p: from a perturbed indicator block, the
    p < 2 stages of pspec_solve and of the lockstep solve end on the components
    with RCut = 0, as the oracle does."""
    from test_oracle_manifold import components_graph
    k = 3
    gs, comps, U0s = [], [], []
    for seed, sizes in ((3, [30, 24, 36]), (4, [300, 240, 410]), (5, [1200, 900, 1500])):
        g, comp = components_graph(sizes, seed)
        g = wl.CSRGraph(g.n, g.rowptr, g.col, g.val.astype(np.float32))
        ind = np.zeros((g.n, k))
        ind[np.arange(g.n), comp] = 1.0
        U0 = oracle.qf(ind + 0.2 * np.random.default_rng(seed).standard_normal(ind.shape)).astype(np.float32)
        gs.append(g), comps.append(comp), U0s.append(U0)
    sched = (1.6, 1.3)
    for g, comp, U0 in zip(gs, comps, U0s):
        S = api.Graph.from_csr(g)
        _, lab, rc, st, _ = S.solve(torch.from_numpy(U0).cuda(), sched, api.default_opts(max_outer=60))
        assert rc == 0.0 and same_partition(lab.cpu().numpy(), comp)
    batch = wl.concat_graphs(gs, [k] * len(gs))
    G = handle(api, batch)
    _, lab, rc, status, stats, _ = G.solve_lockstep(torch.from_numpy(np.concatenate(U0s)).cuda(), sched,
                                                    api.default_opts(max_outer=60))
    for i, comp in enumerate(comps):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        assert rc[i] == 0.0 and same_partition(lab[a:b].cpu().numpy(), comp), i


def test_lockstep_with_hub_rows(api):
    """A graph with a hub row (a star centre joined to 400 vertices; its row
    is split into chunks whose partial sums the last chunk adds) beside
    ordinary ones: its chunk tasks are left out together with the rest of its
    graph, and its p = 2 stage reaches the Laplacian eigenvalue sum as
    pspec_solve on the graph alone does.  (Whether an FP32 stage stops at
    gtol_rel or at its noise floor is decided by rounding, so the comparison
    is on values, not step counts.)"""
    k = 4
    rng = np.random.default_rng(12)
    base = wl.sbm_sampled(rng, 3000, 4, 10.0, 0.9)
    rows = np.repeat(np.arange(base.n), np.diff(base.rowptr))
    ring = np.arange(base.n)
    star = rng.choice(np.arange(1, base.n), 400, replace=False)
    a = np.concatenate([rows, ring, np.zeros(400, np.int64)])
    b = np.concatenate([base.col.astype(np.int64), (ring + 1) % base.n, star])
    w = np.concatenate([base.val.astype(np.float64), np.full(base.n, 0.5), np.full(400, 0.5)])
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    e, first = np.unique(np.stack([lo, hi], 1), axis=0, return_index=True)
    hub = wl.csr_from_undirected(base.n, e[:, 0], e[:, 1], w[first], np.float32)
    assert hub.rowptr[1] - hub.rowptr[0] > 256  # the star centre is split into chunks
    gs = [wl.sbm_sampled(rng, 900, 4, 9.0, 0.9), hub, wl.sbm_sampled(rng, 400, 4, 8.0, 0.9)]
    batch = wl.concat_graphs(gs, [k] * len(gs))
    U = np.concatenate([wl.orthonormal_block(80 + i, g.n, k) for i, g in enumerate(gs)])
    G = handle(api, batch)
    opts = api.default_opts(max_outer=60)
    _, _, rc, status, stats, _ = G.solve_lockstep(torch.from_numpy(U).cuda(), [2.0, 1.6], opts)
    assert all(s in (0, 6) for s in status), status
    for i, g in enumerate(gs):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        S = api.Graph.from_csr(g)
        _, _, rci, sti, _ = S.solve(torch.from_numpy(U[a:b]).cuda(), [2.0, 1.6], opts)
        ev = laplacian_eigs(g, k).sum()
        assert abs(stats[i]["f"][0] - ev) <= 1e-5 * ev, (i, stats[i]["f"][0], ev)
        assert abs(stats[i]["f"][0] - sti["f"][0]) <= 1e-5 * ev, (i, stats[i]["f"][0], sti["f"][0])
        assert abs(rc[i] - rci) <= 0.02 * rci, (i, rc[i], rci)


def test_lockstep_nan_start_stops_only_its_graph(api):
    """A NaN in one graph's starting block is reported for that graph
    (NONFINITE, RCut NaN) at its first evaluation; the other graphs' solves are
    those they have alone."""
    rng = np.random.default_rng(19)
    gs = [wl.sbm_sampled(rng, 500, 3, 9.0, 0.9), wl.sbm_sampled(rng, 700, 3, 9.0, 0.9),
          wl.sbm_sampled(rng, 300, 3, 9.0, 0.9)]
    batch = wl.concat_graphs(gs, [3] * len(gs))
    G = handle(api, batch)
    U = np.concatenate([wl.orthonormal_block(30 + i, g.n, 3) for i, g in enumerate(gs)])
    U[batch.node_off[1] + 17, 2] = np.nan
    _, _, rc, status, stats, st = G.solve_lockstep(torch.from_numpy(U).cuda(), [2.0, 1.7], allow_errors=True)
    assert status[1] == api._abi.PSPEC_ERR_NONFINITE and math.isnan(rc[1])
    assert st == api._abi.PSPEC_ERR_NONFINITE
    for i in (0, 2):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        _, _, rci, sti, _ = api.Graph.from_csr(gs[i]).solve(torch.from_numpy(U[a:b]).cuda(), [2.0, 1.7])
        assert status[i] in (0, 6)
        assert abs(stats[i]["f"][0] - sti["f"][0]) <= 1e-5 * sti["f"][0]
        assert abs(rc[i] - rci) <= 0.01 * rci


def test_sbm_batch_full_size_lockstep_against_per_graph_solves(api):
    """The 512-graph workload (one handle per k): the lockstep solve against
    the per-graph solves of pspec_solve_batched (each equal to pspec_solve
    alone).  Both are FP32 solves whose reductions sum in different orders,
    and most stages end at the Newton cap, so graphs may end on different
    local minima: most RCuts agree to 1% and the median difference is below
    0.1%; every graph ends OK or at the cap in both."""
    batch = wl.make_graph("sbm_batch")
    sched = list(wl.WORKLOADS["sbm_batch"]["p_schedule"])
    rel = []
    for k in (2, 4, 8):
        idx = np.flatnonzero(np.asarray(batch.k) == k)
        gs = [batch.graphs[i] for i in idx]
        sub = wl.concat_graphs(gs, [k] * len(gs))
        G = handle(api, sub)
        U0 = torch.from_numpy(np.concatenate([wl.orthonormal_block(2000 + 10 * k + i, g.n, k)
                                              for i, g in enumerate(gs)])).cuda()
        _, lab, rc, status, _, _ = G.solve_lockstep(U0, sched, api.default_opts(), allow_errors=True)
        _, labb, rcb, statusb, _ = G.solve_batched(U0, sched, api.default_opts())
        assert np.isin(status, (0, 6)).all() and np.isin(statusb, (0, 6)).all()
        # (a graph whose clusters are its components has RCut 0 in both)
        rel.append(np.abs(rc - rcb) / np.where(rcb > 0, rcb, 1.0))
        # the RCut reported is the cut of the labels returned (sampled graphs)
        for i in range(0, len(gs), 17):
            a, b = sub.node_off[i], sub.node_off[i + 1]
            assert abs(rc[i] - oracle.rcut(gs[i], lab[a:b].cpu().numpy(), k)) <= 1e-12 * rc[i]
    rel = np.concatenate(rel)
    assert rel.size == 512
    assert np.median(rel) < 1e-3 and np.mean(rel <= 0.01) >= 0.85, (np.median(rel), np.mean(rel <= 0.01))
