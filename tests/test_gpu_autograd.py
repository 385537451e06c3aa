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


def kink_free_direction(g, U64, V, h):
    """V with its entries zeroed wherever a step of size h along it would carry
    an edge difference u_i - u_j or a vertex value u_i across zero, where F is
    not smooth (|t|^p); zeroing is repeated until no entry crosses, so central
    differences of F along the result see a smooth function."""
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    col = g.col.astype(np.int64)
    V = V / np.linalg.norm(V)  # unit step; the margin 2 covers the renormalisation
    for l in range(V.shape[1]):
        u = np.ascontiguousarray(U64[:, l])
        v = np.ascontiguousarray(V[:, l])
        ad = np.abs(u[rows] - u[col])
        while True:
            # strict: an entry that does not move (zero step) cannot cross
            bad = ad < 2.0 * h * np.abs(v[rows] - v[col])
            badv = np.abs(u) < 2.0 * h * np.abs(v)
            if not bad.any() and not badv.any():
                break
            v[rows[bad]] = 0.0
            v[col[bad]] = 0.0
            v[badv] = 0.0
        V[:, l] = v
    return V / np.linalg.norm(V)


@pytest.mark.slow
def test_dcsbm_autograd_against_oracle(mods):
    """n = 1,000,000, 16 blocks, power-law degrees, k = 16, p = 1.3: the FP32
    autograd gradient against the oracle's, entry by entry; its directional
    derivative against Richardson-extrapolated central differences of the
    oracle's F (h = 1e-3 and 5e-4, FP64) along a direction on which no edge
    difference changes sign inside the stencil; the double backward against
    the oracle's Hessian product on sampled rows (hubs included)."""
    import oracle_rows as orw
    from gpu_common import rel_elem
    api, ag = mods
    g = wl.make_graph("dcsbm")
    G = api.Graph.from_csr(g)
    k, p, h = 16, 1.3, 1e-3
    U0, _ = wl.make_blocks("dcsbm", g.n, k)
    U64 = U0.astype(np.float64)
    U = torch.from_numpy(U0).cuda().requires_grad_(True)
    F = ag.p_objective(U, G, p)
    (gr,) = torch.autograd.grad(F, U, create_graph=True)
    V32 = torch.from_numpy(wl.gaussian_block(78, g.n, k)).cuda()
    (hv,) = torch.autograd.grad(gr, U, grad_outputs=V32)
    torch.cuda.synchronize()
    N, D = orw.oracle_N_D(g, U64, p)
    assert abs(F.item() - np.sum(N / D)) <= 1e-5 * np.sum(N / D)
    delta = orw.oracle_delta(g, U64, p)
    gr_ref = orw.oracle_grad(g, U64, p, N, D, delta)
    got = gr.detach().cpu().numpy()
    assert rel_col(got, gr_ref) <= 1e-5
    assert rel_elem(got, gr_ref, orw.grad_scale(g, U64, p, N, D)) <= 1e-5
    # directional derivative against central differences of the oracle's F
    Vd = kink_free_direction(g, U64, wl.gaussian_block(77, g.n, k, dtype=np.float64), h)

    def F_oracle(X):
        Nx, Dx = orw.oracle_N_D(g, X, p, rows_per_chunk=250_000)
        return float(np.sum(Nx / Dx))

    def central(step):
        return (F_oracle(U64 + step * Vd) - F_oracle(U64 - step * Vd)) / (2 * step)

    fd = (4 * central(h / 2) - central(h)) / 3  # Richardson: error O(h^4)
    dd_ref = float(np.sum(gr_ref * Vd))
    dd = float(np.sum(got.astype(np.float64) * Vd))
    assert abs(dd_ref - fd) <= 1e-6 * abs(fd)  # the oracle's gradient and its F agree
    assert abs(dd - fd) <= 1e-4 * abs(fd)
    # double backward: the Hessian product on sampled rows
    rng = np.random.default_rng(5)
    deg = np.diff(g.rowptr)
    rows = np.unique(np.concatenate([rng.choice(g.n, 300, replace=False),
                                     np.argsort(deg, kind="stable")[-20:]]))
    ref = orw.oracle_hvp_rows(g, U64, V32.cpu().numpy().astype(np.float64), p, rows, N, D, delta)
    assert rel_col(hv.cpu().numpy()[rows], ref) <= 1e-4
