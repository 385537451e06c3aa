"""F_p as a torch.autograd.Function: backward is the gradient kernel and
double backward the Hessian-vector-product kernel, checked by torch's
finite-difference gradcheck/gradgradcheck in FP64, by central differences on
the 1,000,000-vertex power-law workload, and against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_common import rel_col
from paper_2605_26975_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_26975_gb300 import build
    build.build()
    from paper_2605_26975_gb300 import api, autograd
    return api, autograd


def tiny_graph():
    rng = np.random.default_rng(0)
    n = 12
    A = np.triu((rng.random((n, n)) < 0.5) * rng.uniform(0.3, 1.5, (n, n)), 1)
    iu, ju = np.nonzero(A)
    return wl.csr_from_undirected(n, iu, ju, A[iu, ju], np.float64)


@pytest.mark.parametrize("p", [2.0, 1.6, 1.2])
def test_gradcheck_and_gradgradcheck_fp64(mods, p):
    api, ag = mods
    g = tiny_graph()
    G = api.Graph.from_csr(g)
    rng = np.random.default_rng(1)
    U0 = rng.permutation(g.n)[:, None] * 0.3 + np.array([[0.05, -0.4]]) + 0.01 * rng.random((g.n, 2))
    U = torch.tensor(U0, dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda X: ag.p_objective(X, G, p)
    assert torch.autograd.gradcheck(f, (U,), eps=1e-6, atol=1e-7, rtol=1e-6)
    assert torch.autograd.gradgradcheck(f, (U,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_backward_matches_oracle_fp32(mods):
    api, ag = mods
    g = wl.make_graph("sbm4")
    G = api.Graph.from_csr(g)
    U0 = wl.orthonormal_block(2000, g.n, 4)
    V0 = wl.gaussian_block(3000, g.n, 4)
    U = torch.from_numpy(U0).cuda().requires_grad_(True)
    F = ag.p_objective(U, G, 1.4)
    (gr,) = torch.autograd.grad(F, U, create_graph=True)
    Vt = torch.from_numpy(V0).cuda()
    (hv,) = torch.autograd.grad(gr, U, grad_outputs=Vt)
    U64, V64 = U0.astype(np.float64), V0.astype(np.float64)
    assert abs(F.item() - oracle.objective(g, U64, 1.4)) <= 1e-5 * F.item()
    assert rel_col(gr.detach().cpu().numpy(), oracle.euclidean_grad(g, U64, 1.4)) <= 1e-5
    assert rel_col(hv.cpu().numpy(), oracle.euclidean_hvp(g, U64, V64, 1.4)) <= 1e-4
    # the double-backward is the HVP kernel itself
    assert torch.equal(hv, G.hvp(U.detach(), Vt, 1.4))


@pytest.mark.slow
def test_dcsbm_autograd_central_differences(mods):
    """n = 1,000,000, 16 blocks, power-law degrees, k = 16, p = 1.3: the FP32
    autograd gradient against central differences of F in FP64 (h = 1e-3, unit
    direction) and the FP64 device gradient; the double backward against the
    FP64 Hessian product."""
    api, ag = mods
    g = wl.make_graph("dcsbm")
    G = api.Graph.from_csr(g)
    k, p, h = 16, 1.3, 1e-3
    U0, _ = wl.make_blocks("dcsbm", g.n, k)
    V0 = wl.gaussian_block(77, g.n, k, dtype=np.float64)
    V0 /= np.linalg.norm(V0)
    U = torch.from_numpy(U0).cuda().requires_grad_(True)
    F = ag.p_objective(U, G, p)
    (gr,) = torch.autograd.grad(F, U, create_graph=True)
    U64 = torch.from_numpy(U0.astype(np.float64)).cuda()
    Vd = torch.from_numpy(V0).cuda()
    Fp, _ = G.eval(U64 + h * Vd, p)
    Fm, _ = G.eval(U64 - h * Vd, p)
    fd = (Fp.item() - Fm.item()) / (2 * h)
    dd = float((gr.double() * Vd).sum())
    _, g64 = G.eval(U64, p)
    dd64 = float((g64 * Vd).sum())
    # the FP32 autograd derivative against the exact FP64 one
    assert abs(dd - dd64) <= 1e-5 * abs(dd64)
    assert rel_col(gr.detach().cpu().numpy(), g64.cpu().numpy()) <= 1e-5
    # central differences: at p = 1.3 the few edges whose difference changes
    # sign inside the +-h stencil (|d| < h |v_i - v_j|, ~1e-4 of the 16M
    # entries) bend F like |t|^p, which bounds the stencil's agreement to ~1e-4
    assert abs(dd64 - fd) <= 1e-3 * abs(fd)
    V32 = torch.from_numpy(wl.gaussian_block(78, g.n, k)).cuda()
    (hv,) = torch.autograd.grad(gr, U, grad_outputs=V32)
    hv64 = G.hvp(U64, V32.double(), p)
    assert rel_col(hv.cpu().numpy(), hv64.cpu().numpy()) <= 1e-4
