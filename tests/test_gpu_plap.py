"""GPU parity of pspec_eval / pspec_hvp against the FP64 oracle.

The oracle receives exactly the FP32 values the GPU receives (U, V and W
widened to float64), so differences come from the kernels' arithmetic only.
"""
import numpy as np
import pytest

import oracle
from gpu_common import (TOL_F64, check_eval, check_hvp, quantised_block, rel_col, small_graphs,
                        tied_heavy_graph)
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


@pytest.fixture(scope="module")
def graphs(api):
    out = {}
    for name, g in small_graphs().items():
        out[name] = (g, api.Graph.from_csr(g))
    return out


def blocks(n, k, seed):
    U = wl.orthonormal_block(seed, n, k, np.float32)
    V = wl.gaussian_block(seed + 1, n, k, dtype=np.float32)
    return U, V


@pytest.mark.parametrize("name", ["sbm", "grid", "knn", "hubs", "isolated"])
@pytest.mark.parametrize("k", [1, 3, 4, 8, 16])
@pytest.mark.parametrize("p", [2.0, 1.5, 1.1])
def test_eval_and_hvp_match_oracle(api, graphs, name, k, p):
    g, G = graphs[name]
    U, V = blocks(g.n, k, 100 + k)
    check_eval(api, g, G, U, p)
    check_hvp(api, g, G, U, V, p)


@pytest.mark.parametrize("k", [2, 5, 6, 7, 9, 10, 11, 12, 13, 14, 15])
def test_every_k(api, graphs, k):
    g, G = graphs["sbm"]
    U, V = blocks(g.n, k, 7 * k)
    check_eval(api, g, G, U, 1.3)
    check_hvp(api, g, G, U, V, 1.3)


@pytest.mark.parametrize("p", [2.0, 1.7, 1.2])
def test_ties_and_zeros(api, graphs, p):
    # quantised values: many exact zero differences and exact zero entries
    g, G = graphs["sbm"]
    rng = np.random.default_rng(9)
    U = (rng.integers(-3, 4, size=(g.n, 4)) * 0.25).astype(np.float32)
    V = rng.standard_normal((g.n, 4)).astype(np.float32)
    check_eval(api, g, G, U, p)
    check_hvp(api, g, G, U, V, p)


@pytest.fixture(scope="module")
def tied_heavy(api):
    g = tied_heavy_graph()
    return g, api.Graph.from_csr(g)


@pytest.mark.parametrize("p", [1.01, 1.05, 1.1, 2.0])
@pytest.mark.parametrize("k", [4, 8, 3])
def test_ties_with_large_weights(api, tied_heavy, p, k):
    """Tied entries (u_i == u_j) under weights up to 1e6: a tie contributes
    phi_p(0) = 0 and, for p < 2, no curvature term, whatever its weight, so
    every result is finite and equals the oracle's (no status raised)."""
    g, G = tied_heavy
    assert g.val.max() > 2.0 ** (128 - 126 * (2 - 1.01))  # beyond FP32 when clamped
    U = quantised_block(40 + k, g.n, k)
    V = wl.gaussian_block(41 + k, g.n, k, dtype=np.float32)
    check_eval(api, g, G, U, p)
    check_hvp(api, g, G, U, V, p)


@pytest.mark.parametrize("k", [1, 4, 8])
def test_plain_fp64_path(api, graphs, k):
    g, G = graphs["hubs"]
    U, V = blocks(g.n, k, 55)
    U64, V64 = U.astype(np.float64), V.astype(np.float64)
    Ud = torch.from_numpy(U64).cuda()
    Vd = torch.from_numpy(V64).cuda()
    for p in (2.0, 1.4):
        F, grad = G.eval(Ud, p)
        HV = G.hvp(Ud, Vd, p)
        torch.cuda.synchronize()
        assert abs(F.item() - oracle.objective(g, U64, p)) <= TOL_F64 * abs(F.item())
        assert rel_col(grad.cpu().numpy(), oracle.euclidean_grad(g, U64, p)) <= TOL_F64
        assert rel_col(HV.cpu().numpy(), oracle.euclidean_hvp(g, U64, V64, p)) <= 1e-10


def test_kept_delta_reuse(api, graphs):
    """pspec_eval(PSPEC_KEEP_DELTA) then pspec_hvp(PSPEC_DELTA_KEPT) at the same
    U: the gradient is bit-identical to the plain call's, the Hessian product
    matches the oracle (and the plain call within rounding), through device
    and host pointers; a kept Delta for another U, k or p is refused."""
    from paper_2605_26975_gb300 import _abi
    g, G = graphs["hubs"]
    U, V = blocks(g.n, 8, 61)
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    for p in (1.3, 2.0, 1.05):
        F1, g1 = G.eval(Ud, p)
        F2, g2 = G.eval(Ud, p, keep_delta=True)
        h_plain = G.hvp(Ud, Vd, p)
        h_kept = G.hvp(Ud, Vd, p, delta_kept=True)
        torch.cuda.synchronize()
        assert G.status() == 0
        assert F1.item() == F2.item() and torch.equal(g1, g2)
        ref = oracle.euclidean_hvp(g, U.astype(np.float64), V.astype(np.float64), p)
        assert rel_col(h_kept.cpu().numpy(), ref) <= 1e-4
        assert rel_col(h_kept.cpu().numpy(), h_plain.cpu().numpy().astype(np.float64)) <= 1e-5
    # host pointers: the same kept rows through PSPEC_HOST_PTRS
    Uh, Vh = torch.from_numpy(U).pin_memory(), torch.from_numpy(V).pin_memory()
    gh, hh = torch.empty_like(Uh).pin_memory(), torch.empty_like(Uh).pin_memory()
    G.eval_host(Uh, 1.3, gh, keep_delta=True)
    G.hvp_host(Uh, Vh, 1.3, hh, delta_kept=True)
    G.eval(Ud, 1.3, keep_delta=True)
    hd = G.hvp(Ud, Vd, 1.3, delta_kept=True)
    torch.cuda.synchronize()
    assert torch.equal(hh, hd.cpu())
    # the kept host-pointer HVP reuses the staged copy of U; a host-pointer
    # call with another U in between must not leak into it
    U2h = torch.from_numpy(blocks(g.n, 8, 62)[0]).pin_memory()
    G.eval_host(Uh, 1.3, gh, keep_delta=True)
    G.hvp_host(Uh, Vh, 1.3, hh, delta_kept=True)
    G.eval_host(U2h, 1.3, torch.empty_like(gh).pin_memory())  # stages U2, keeps nothing new
    h2 = torch.empty_like(hh).pin_memory()
    G.hvp_host(Uh, Vh, 1.3, h2, delta_kept=True)  # Uh's kept record still stands
    assert torch.equal(h2, hd.cpu()) and torch.equal(hh, hd.cpu())
    # refused: another p, another U pointer, another k, the host flag, FP64
    G.eval(Ud, 1.3, keep_delta=True)  # the last kept point: a device-pointer call
    with pytest.raises(_abi.PspecError):
        G.hvp(Ud, Vd, 1.7, delta_kept=True)
    with pytest.raises(_abi.PspecError):
        G.hvp(Ud.clone(), Vd, 1.3, delta_kept=True)
    with pytest.raises(_abi.PspecError):
        G.hvp(Ud[:, :4].contiguous(), Vd[:, :4].contiguous(), 1.3, delta_kept=True)
    with pytest.raises(_abi.PspecError):
        G.hvp_host(Uh, Vh, 1.3, hh, delta_kept=True)  # kept by a device-pointer call
    with pytest.raises(_abi.PspecError):
        G.eval(Ud.double(), 1.3, keep_delta=True)


def test_bit_reproducible(api, graphs):
    g, G = graphs["hubs"]
    U, V = blocks(g.n, 8, 77)
    Ud = torch.from_numpy(U).cuda()
    Vd = torch.from_numpy(V).cuda()
    F1, g1 = G.eval(Ud, 1.3)
    h1 = G.hvp(Ud, Vd, 1.3)
    F2, g2 = G.eval(Ud, 1.3)
    h2 = G.hvp(Ud, Vd, 1.3)
    torch.cuda.synchronize()
    assert F1.item() == F2.item()
    assert torch.equal(g1, g2) and torch.equal(h1, h2)


def test_host_pointer_path_matches_device(api, graphs):
    g, G = graphs["knn"]
    U, V = blocks(g.n, 8, 31)
    Uh = torch.from_numpy(U).pin_memory()
    Vh = torch.from_numpy(V).pin_memory()
    gh = torch.empty_like(Uh).pin_memory()
    hh = torch.empty_like(Uh).pin_memory()
    F_host = G.eval_host(Uh, 1.5, gh)
    G.hvp_host(Uh, Vh, 1.5, hh)
    F, grad = G.eval(Uh.cuda(), 1.5)
    HV = G.hvp(Uh.cuda(), Vh.cuda(), 1.5)
    torch.cuda.synchronize()
    assert F_host == F.item()
    assert torch.equal(gh, grad.cpu()) and torch.equal(hh, HV.cpu())


def test_single_vertex_and_empty_graph(api):
    g = wl.CSRGraph(1, np.array([0, 0], dtype=np.int64), np.zeros(0, np.int32),
                    np.zeros(0, np.float32))
    G = api.Graph.from_csr(g)
    U = torch.tensor([[0.7]], device="cuda")
    F, grad = G.eval(U, 1.5)
    HV = G.hvp(U, torch.tensor([[1.0]], device="cuda"), 1.5)
    torch.cuda.synchronize()
    assert F.item() == 0.0
    assert grad.item() == 0.0
    ref = oracle.euclidean_hvp(g, np.array([[0.7]]), np.array([[1.0]]), 1.5)
    assert abs(HV.item() - ref[0, 0]) <= 1e-5 * abs(ref[0, 0])


def test_zero_column_and_nonfinite_are_reported(api, graphs):
    from paper_2605_26975_gb300 import _abi
    g, G = graphs["sbm"]
    U, _ = blocks(g.n, 4, 3)
    U[:, 2] = 0.0
    G.eval(torch.from_numpy(U).cuda(), 1.5)
    assert G.status() == _abi.PSPEC_ERR_ZERO_COLUMN
    U, _ = blocks(g.n, 4, 3)
    U[10, 1] = np.nan
    G.eval(torch.from_numpy(U).cuda(), 1.5)
    assert G.status() == _abi.PSPEC_ERR_NONFINITE
    # the status word is cleared once read
    U, _ = blocks(g.n, 4, 3)
    G.eval(torch.from_numpy(U).cuda(), 1.5)
    assert G.status() == 0


def test_invalid_arguments(api, graphs):
    from paper_2605_26975_gb300 import _abi
    g, G = graphs["sbm"]
    U = torch.zeros((g.n, 4), device="cuda")
    for p in (1.0, 2.5, float("nan")):
        with pytest.raises(_abi.PspecError):
            G.eval(U, p)
    with pytest.raises(_abi.PspecError):
        G.eval(torch.zeros((g.n, 17), device="cuda"), 1.5)
    # misaligned block: a view that starts one float into a 16-byte-aligned buffer
    buf = torch.zeros(g.n * 4 + 1, device="cuda")
    with pytest.raises(_abi.PspecError):
        G.eval(buf[1:].view(g.n, 4), 1.5)


@pytest.mark.parametrize("k", [4, 8, 16])
def test_staged_kernel_parity(api, k, monkeypatch):
    """The staged (cp.async) edge kernel, which runs when a task's entries fit
    its buffers (here 8 entries per lane, set through PSPEC_EDGES_PER_LANE;
    the default shape runs the direct kernel): F, gradient, the Hessian
    product and the kept-point Hessian product against the oracle, on a graph
    with hub rows and on one with heavy weights and exact ties."""
    from gpu_common import TOL_HVP, star_plus_powerlaw
    monkeypatch.setenv("PSPEC_EDGES_PER_LANE", "8")
    cases = [(star_plus_powerlaw(seed=11, n=4000), lambda n: wl.orthonormal_block(41, n, k)),
             (tied_heavy_graph(3, 2000), lambda n: quantised_block(43, n, k))]
    for g, make_u in cases:
        G = api.Graph.from_csr(g)
        U = make_u(g.n)
        V = wl.gaussian_block(42, g.n, k)
        for p in (1.3, 2.0):
            check_eval(api, g, G, U, p)
            check_hvp(api, g, G, U, V, p)
            Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
            G.eval(Ud, p, keep_delta=True)
            HVk = G.hvp(Ud, Vd, p, delta_kept=True)
            torch.cuda.synchronize()
            ref = oracle.euclidean_hvp(g, U.astype(np.float64), V.astype(np.float64), p)
            assert rel_col(HVk.cpu().numpy(), ref) <= TOL_HVP
