"""pspec_tune: the launch-shape autotuner of the edge kernels.  It must report
every candidate with a positive time, keep the fastest, and leave the handle
computing the same F, gradient and HVP (parity with the FP64 oracle) with
the chosen shape, for single and batched handles."""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_F, TOL_GRAD, TOL_HVP, rel_col, star_plus_powerlaw
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


def parity(G, g, U, V, p):
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    F, grad = G.eval(Ud, p)
    HV = G.hvp(Ud, Vd, p)
    torch.cuda.synchronize()
    assert G.status() == 0
    U64, V64 = U.astype(np.float64), V.astype(np.float64)
    F_ref = oracle.objective(g, U64, p)
    assert abs(F.item() - F_ref) <= TOL_F * F_ref
    assert rel_col(grad.cpu().numpy(), oracle.euclidean_grad(g, U64, p)) <= TOL_GRAD
    assert rel_col(HV.cpu().numpy(), oracle.euclidean_hvp(g, U64, V64, p)) <= TOL_HVP
    return F, grad, HV


@pytest.mark.parametrize("k", [3, 8, 16])
def test_tune_keeps_fastest_and_parity(api, k):
    g = star_plus_powerlaw(seed=9, n=30_000)
    G = api.Graph.from_csr(g)
    U = wl.orthonormal_block(21, g.n, k)
    V = wl.gaussian_block(22, g.n, k)
    p = 1.4
    cands, chosen = G.tune(torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), p, reps=3)
    assert len(cands) >= 5
    assert all(ms > 0 for _, _, ms in cands)
    Ls = sorted({L for L, _, _ in cands})
    assert len(Ls) == 5 and all(b == 2 * a for a, b in zip(Ls, Ls[1:]))
    assert chosen == int(np.argmin([ms for _, _, ms in cands]))
    F1, g1, H1 = parity(G, g, U, V, p)
    # the chosen shape is kept: repeated calls are bit-identical
    F2, g2, H2 = parity(G, g, U, V, p)
    assert torch.equal(F1, F2) and torch.equal(g1, g2) and torch.equal(H1, H2)


def test_tune_batched(api):
    rng = np.random.default_rng(3)
    gs = [wl.sbm_sampled(rng, n, 3, 10.0, 0.9) for n in (900, 4000, 150, 2500)]
    batch = wl.concat_graphs(gs, [4] * len(gs))
    c = batch.csr
    G = api.Graph(c.rowptr, c.col, c.val, node_off=batch.node_off)
    k, p = 4, 1.5
    U = np.concatenate([wl.gaussian_block(30 + i, gi.n, k) for i, gi in enumerate(gs)])
    V = np.concatenate([wl.gaussian_block(60 + i, gi.n, k) for i, gi in enumerate(gs)])
    cands, chosen = G.tune(torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), p, reps=2)
    assert 0 <= chosen < len(cands)
    F, grad = G.eval(torch.from_numpy(U).cuda(), p)
    HV = G.hvp(torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), p)
    assert G.status() == 0
    for i, gi in enumerate(gs):
        a, b = batch.node_off[i], batch.node_off[i + 1]
        U64, V64 = U[a:b].astype(np.float64), V[a:b].astype(np.float64)
        assert abs(F[i].item() - oracle.objective(gi, U64, p)) <= TOL_F * oracle.objective(gi, U64, p)
        assert rel_col(grad[a:b].cpu().numpy(), oracle.euclidean_grad(gi, U64, p)) <= TOL_GRAD
        assert rel_col(HV[a:b].cpu().numpy(), oracle.euclidean_hvp(gi, U64, V64, p)) <= TOL_HVP


def test_tune_rejects_bad_arguments(api):
    g = star_plus_powerlaw(seed=9, n=2000)
    G = api.Graph.from_csr(g)
    U = torch.from_numpy(wl.orthonormal_block(1, g.n, 4)).cuda()
    with pytest.raises(api._abi.PspecError):
        G.tune(U, U, 2.5)
    with pytest.raises(api._abi.PspecError):
        G.tune(U, U, 1.5, reps=0)
