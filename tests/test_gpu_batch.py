"""GPU parity of batched handles (pspec_graph_create_batched): every graph of
the concatenation is its own problem, with its own F, N_l, D_l, lambda_l and
rank-two Hessian terms, evaluated in one launch over the concatenated CSR.

Each graph's slice of the batched results is compared with the FP64 oracle
run on that graph alone, on the same FP32 inputs.
"""
import numpy as np
import pytest

import oracle
from gpu_common import (TOL_F, TOL_GRAD, TOL_HVP, grad_term_scale, hvp_term_scale, rel_col, rel_terms,
                        star_plus_powerlaw, with_isolated)
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


def edgeless(n):
    return wl.csr_from_undirected(n, np.zeros(0, np.int64), np.zeros(0, np.int64),
                                  np.zeros(0), np.float32)


def mixed_batch():
    """Ragged sizes, a hub-heavy graph, isolated vertices, a single edge and a
    graph with no edges at all."""
    rng = np.random.default_rng(11)
    gs = [wl.sbm_sampled(rng, 700, 3, 9.0, 0.9),
          star_plus_powerlaw(seed=5, n=6000),
          wl.sbm_sampled(rng, 37, 2, 5.0, 0.9),
          with_isolated(seed=6, n=1500),
          wl.csr_from_undirected(2, np.array([0]), np.array([1]), np.array([0.75]), np.float32),
          edgeless(5),
          wl.knn_gaussian_mixture(8, n=2500, mixtures=3)]
    return wl.concat_graphs(gs, [0] * len(gs))


def batch_blocks(batch, k, seed):
    U = np.concatenate([wl.gaussian_block(seed + i, g.n, k) for i, g in enumerate(batch.graphs)])
    V = np.concatenate([wl.gaussian_block(seed + 500 + i, g.n, k) for i, g in enumerate(batch.graphs)])
    return U, V


def handle(api, batch):
    c = batch.csr
    return api.Graph(c.rowptr, c.col, c.val, node_off=batch.node_off)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16])
@pytest.mark.parametrize("p", [2.0, 1.5, 1.1])
def test_batched_eval_hvp_per_graph_oracle(api, k, p):
    batch = mixed_batch()
    G = handle(api, batch)
    assert G.n_graphs == len(batch.graphs)
    U, V = batch_blocks(batch, k, 40)
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    F, grad, parts = G.eval(Ud, p, parts=True)
    HV = G.hvp(Ud, Vd, p)
    torch.cuda.synchronize()
    assert G.status() == 0
    F, grad, HV = F.cpu().numpy(), grad.cpu().numpy(), HV.cpu().numpy()
    P = parts.cpu().numpy().reshape(-1, 2 * k)
    for i, g in enumerate(batch.graphs):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        U64, V64 = U[a:b].astype(np.float64), V[a:b].astype(np.float64)
        N, D = oracle.objective_parts(g, U64, p)
        F_ref = oracle.objective(g, U64, p)
        assert abs(F[i] - F_ref) <= TOL_F * abs(F_ref) + 1e-300, (i, F[i], F_ref)
        assert np.allclose(P[i, :k], N, rtol=TOL_F, atol=1e-30)
        assert np.allclose(P[i, k:], D, rtol=TOL_F, atol=0)
        # against the magnitude of the terms: the 2-vertex graph's columns
        # cancel to a few percent of their terms
        assert rel_terms(grad[a:b], oracle.euclidean_grad(g, U64, p),
                         grad_term_scale(oracle, g, U64, p)) <= TOL_GRAD, i
        assert rel_terms(HV[a:b], oracle.euclidean_hvp(g, U64, V64, p),
                         hvp_term_scale(oracle, g, U64, V64, p)) <= TOL_HVP, i
        if g.n >= 30:
            assert rel_col(grad[a:b], oracle.euclidean_grad(g, U64, p)) <= TOL_GRAD, i
            assert rel_col(HV[a:b], oracle.euclidean_hvp(g, U64, V64, p)) <= TOL_HVP, i


def test_batched_matches_single_handles_and_is_deterministic(api):
    batch = mixed_batch()
    G = handle(api, batch)
    k, p = 8, 1.3
    U, V = batch_blocks(batch, k, 70)
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    F1, g1 = G.eval(Ud, p)
    F2, g2 = G.eval(Ud, p)
    H1, H2 = G.hvp(Ud, Vd, p), G.hvp(Ud, Vd, p)
    assert torch.equal(F1, F2) and torch.equal(g1, g2) and torch.equal(H1, H2)
    for i, g in enumerate(batch.graphs):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        S = api.Graph.from_csr(g)
        Fs, gs = S.eval(Ud[a:b].contiguous(), p)
        Hs = S.hvp(Ud[a:b].contiguous(), Vd[a:b].contiguous(), p)
        assert abs(F1[i].item() - Fs.item()) <= 2 * TOL_F * abs(Fs.item())
        if g.n >= 30:
            assert rel_col(g1[a:b].cpu().numpy(), gs.cpu().numpy().astype(np.float64)) <= 2 * TOL_GRAD
            assert rel_col(H1[a:b].cpu().numpy(), Hs.cpu().numpy().astype(np.float64)) <= 2 * TOL_HVP


def test_batched_host_pointers(api):
    batch = mixed_batch()
    G = handle(api, batch)
    k, p = 4, 1.6
    U, _ = batch_blocks(batch, k, 90)
    Uh = torch.from_numpy(U).pin_memory()
    gh = torch.empty_like(Uh).pin_memory()
    F = G.eval_host(Uh, p, gh)
    Fd, gd = G.eval(Uh.cuda(), p)
    assert np.array_equal(np.array(F), Fd.cpu().numpy())
    assert torch.equal(gh, gd.cpu())


def test_batched_rejects_fp64(api):
    batch = mixed_batch()
    G = handle(api, batch)
    U, _ = batch_blocks(batch, 4, 1)
    with pytest.raises(api._abi.PspecError):
        G.eval(torch.from_numpy(U.astype(np.float64)).cuda(), 1.5)


def test_batched_zero_column_flagged_per_graph(api):
    """A column that vanishes on one graph of the batch (D = 0 there) raises
    ZERO_COLUMN through the status word; the other graphs stay finite."""
    batch = mixed_batch()
    G = handle(api, batch)
    U, _ = batch_blocks(batch, 2, 3)
    a, b = batch.node_off[2], batch.node_off[3]
    U[a:b, 1] = 0.0
    F, _ = G.eval(torch.from_numpy(U).cuda(), 1.5)
    assert G.status() == api._abi.PSPEC_ERR_ZERO_COLUMN
    Fh = F.cpu().numpy()
    assert np.isfinite(np.delete(Fh, 2)).all()


@pytest.mark.slow
def test_sbm_batch_full_size_sampled(api):
    """The 512-graph workload (about 5.5M vertices, 77M stored entries), one
    handle per k in {2, 4, 8}: every graph's F against the FP64 oracle, and
    gradient / HVP rows of a sample of graphs."""
    batch = wl.make_graph("sbm_batch")
    p = 1.2
    rng = np.random.default_rng(0)
    for k in (2, 4, 8):
        idx = np.flatnonzero(batch.k == k)
        sub = wl.concat_graphs([batch.graphs[i] for i in idx], [k] * idx.size)
        G = handle(api, sub)
        U, V = batch_blocks(sub, k, 2004)
        Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
        F, grad = G.eval(Ud, p)
        HV = G.hvp(Ud, Vd, p)
        torch.cuda.synchronize()
        assert G.status() == 0
        F = F.cpu().numpy()
        for j, g in enumerate(sub.graphs):
            a, b = sub.node_off[j], sub.node_off[j + 1]
            F_ref = oracle.objective(g, U[a:b].astype(np.float64), p)
            assert abs(F[j] - F_ref) <= TOL_F * F_ref, (k, j)
        for j in rng.choice(len(sub.graphs), size=4, replace=False):
            g = sub.graphs[j]
            a, b = sub.node_off[j], sub.node_off[j + 1]
            U64, V64 = U[a:b].astype(np.float64), V[a:b].astype(np.float64)
            assert rel_col(grad[a:b].cpu().numpy(), oracle.euclidean_grad(g, U64, p)) <= TOL_GRAD
            assert rel_col(HV[a:b].cpu().numpy(), oracle.euclidean_hvp(g, U64, V64, p)) <= TOL_HVP
