"""pspec_hvp_noalloc, the allocation-free Hessian-vector product for callers
that cannot allocate device memory (memory owned by another runtime's
allocator, code that must not enter cudaMalloc), against pspec_hvp on the
same inputs and against the FP64 oracle.

Every case calls the entry point through the C ABI twice in a row with
different inputs: the second call reuses the library's fixed working array,
so it also checks that nothing from the first call leaks into the second.
The cases cover the size limit (n * k = 524288, which with k = 1 runs the
block cap and the grid-stride loop), the widest rows (k = 16), p = 2 (no
zero rule) and tied entries under weights up to 1e6.  The file is named so
that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

import oracle
from gpu_common import TOL_HVP, quantised_block, rel_col, tied_heavy_graph
from paper_2605_26975_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LIMIT = 1 << 19  # n * k limit of the static working array


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_26975_gb300 import _abi, build
    build.build()
    return _abi


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _noalloc(abi, g_dev, U, V, p, out):
    rowptr, col, val = g_dev
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return abi.lib().pspec_hvp_noalloc(U.shape[0], _ptr(rowptr), _ptr(col), _ptr(val), _ptr(U),
                                       _ptr(V), U.shape[1], p, _ptr(out), stream)


def _graph(kind, n):
    if kind == "tied_heavy":
        return tied_heavy_graph(n=n)
    return wl.sbm_sampled(np.random.default_rng(21), n, 4, 12.0, 0.85)


# (graph, n, k, [(block seed, p) of the two calls])
CASES = [
    ("sbm", 4000, 4, [(1, 1.4), (2, 1.15)]),
    ("sbm", 4000, 8, [(1, 1.4), (2, 1.15)]),
    ("sbm", 4000, 3, [(1, 1.4), (2, 1.15)]),
    ("sbm", LIMIT, 1, [(3, 1.3), (4, 1.6)]),
    ("sbm", LIMIT // 16, 16, [(5, 1.2), (6, 1.5)]),
    ("sbm", 4000, 8, [(7, 2.0), (8, 2.0)]),
    ("tied_heavy", 3000, 4, [(9, 1.01), (10, 1.1)]),
]


@pytest.mark.parametrize("kind,n,k,calls", CASES,
                         ids=[f"{c[0]}-n{c[1]}-k{c[2]}-p{c[3][0][1]}" for c in CASES])
def test_noalloc_matches_pspec_hvp_and_oracle_twice(lib, kind, n, k, calls):
    from paper_2605_26975_gb300 import api
    g = _graph(kind, n)
    G = api.Graph.from_csr(g)
    g_dev = (torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(),
             torch.from_numpy(g.val).cuda())
    for call, (seed, p) in enumerate(calls):
        if kind == "tied_heavy":
            U = torch.from_numpy(quantised_block(seed, g.n, k)).cuda()
        else:
            U = torch.from_numpy(wl.orthonormal_block(seed, g.n, k)).cuda()
        V = torch.from_numpy(wl.gaussian_block(seed + 50, g.n, k)).cuda()
        ref = G.hvp(U, V, p)
        out = torch.full_like(U, float("nan"))
        assert _noalloc(lib, g_dev, U, V, p, out) == lib.PSPEC_OK, lib.lib().pspec_last_error()
        torch.cuda.synchronize()
        assert G.status() == 0
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert rel_col(got, ref.cpu().numpy().astype(np.float64)) <= TOL_HVP, call
        exact = oracle.euclidean_hvp(g, U.cpu().numpy().astype(np.float64),
                                     V.cpu().numpy().astype(np.float64), p)
        assert rel_col(got, exact) <= TOL_HVP, call


def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    n, k = LIMIT // 8 + 1, 8
    dummy = torch.zeros(8, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = lib.lib().pspec_hvp_noalloc(n, p, p, p, p, p, k, 1.5, p, None)
    assert st == lib.PSPEC_ERR_INVALID_ARG
    assert b"524288" in lib.lib().pspec_last_error()
