"""pspec_solve_batched: every graph of a batched handle solved as its own
problem, concurrently.  Each graph's result must equal pspec_solve on that
graph alone (same kernels, same order on the graph's own stream), and the
1,000-vertex SBM inside a batch must match the FP64 oracle's solve."""
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


def batch_and_blocks(k):
    rng = np.random.default_rng(21)
    gs = [wl.make_graph("sbm4"),
          wl.sbm_sampled(rng, 3000, 4, 12.0, 0.9),
          wl.sbm_sampled(rng, 200, 3, 8.0, 0.9),
          wl.knn_gaussian_mixture(4, n=5000, mixtures=4)]
    batch = wl.concat_graphs(gs, [k] * len(gs))
    U = np.concatenate([wl.orthonormal_block(2000 if i == 0 else 500 + i, g.n, k)
                        for i, g in enumerate(gs)])
    return gs, batch, U


def test_batched_solve_equals_single_solves(api):
    k = 4
    sched = (2.0, 1.6, 1.3)
    gs, batch, U = batch_and_blocks(k)
    c = batch.csr
    G = api.Graph(c.rowptr, c.col, c.val, node_off=batch.node_off)
    Ub, lab, rc, status, st = G.solve_batched(torch.from_numpy(U).cuda(), sched, threads=4)
    assert all(s in (0, 6) for s in status)  # OK or NOT_CONVERGED
    for i, g in enumerate(gs):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        S = api.Graph.from_csr(g)
        Ui, labi, rci, _, _ = S.solve(torch.from_numpy(U[a:b]).cuda(), sched)
        assert torch.equal(Ub[a:b], Ui), i
        assert torch.equal(lab[a:b], labi), i
        assert rc[i] == rci, i
    # a second call reuses the per-graph handles and gives the same result
    Ub2, lab2, rc2, _, _ = G.solve_batched(torch.from_numpy(U).cuda(), sched, threads=2)
    assert torch.equal(Ub, Ub2) and torch.equal(lab, lab2) and np.array_equal(rc, rc2)


def test_batched_solve_sbm4_matches_oracle(api):
    k = 4
    sched = wl.WORKLOADS["sbm4"]["p_schedule"]
    gs, batch, U = batch_and_blocks(k)
    c = batch.csr
    G = api.Graph(c.rowptr, c.col, c.val, node_off=batch.node_off)
    Ub, lab, rc, status, st = G.solve_batched(torch.from_numpy(U).cuda(), sched)
    n0 = gs[0].n
    _, ref_lab, ref_rc, _ = oracle.solve(gs[0], U[:n0].astype(np.float64), sched)
    assert abs(rc[0] - ref_rc) <= 0.01 * ref_rc
    assert same_partition(lab[:n0].cpu().numpy(), ref_lab)


def test_batched_solve_reports_a_graph_smaller_than_k(api):
    rng = np.random.default_rng(5)
    gs = [wl.sbm_sampled(rng, 400, 2, 8.0, 0.9),
          wl.csr_from_undirected(2, np.array([0]), np.array([1]), np.array([1.0]), np.float32)]
    batch = wl.concat_graphs(gs, [3, 3])
    c = batch.csr
    G = api.Graph(c.rowptr, c.col, c.val, node_off=batch.node_off)
    U = np.concatenate([wl.gaussian_block(i, g.n, 3) for i, g in enumerate(gs)])
    with pytest.raises(api._abi.PspecError, match="graph 1"):
        G.solve_batched(torch.from_numpy(U).cuda(), [2.0])
