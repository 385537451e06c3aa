"""pspec_hvp_noalloc, the allocation-free Hessian-vector product for callers
that cannot allocate device memory, against pspec_hvp on the same inputs.

Called through the C ABI twice in a row: the second call reuses the
library's fixed working array, so it also checks that nothing from the first
call leaks into the second.  The file is named so that pytest collects it
last."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import TOL_HVP, rel_col
from paper_2605_26975_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


@pytest.mark.parametrize("k", [4, 8, 3])
def test_noalloc_matches_pspec_hvp_twice(lib, k):
    from paper_2605_26975_gb300 import api
    g = wl.sbm_sampled(np.random.default_rng(21), 4000, 4, 12.0, 0.85)
    G = api.Graph.from_csr(g)
    g_dev = (torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(),
             torch.from_numpy(g.val).cuda())
    for call, (seed, p) in enumerate([(1, 1.4), (2, 1.15)]):
        U = torch.from_numpy(wl.orthonormal_block(seed, g.n, k)).cuda()
        V = torch.from_numpy(wl.gaussian_block(seed + 50, g.n, k)).cuda()
        ref = G.hvp(U, V, p)
        out = torch.full_like(U, float("nan"))
        assert _noalloc(lib, g_dev, U, V, p, out) == lib.PSPEC_OK, lib.lib().pspec_last_error()
        torch.cuda.synchronize()
        assert rel_col(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= TOL_HVP, call


def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    n, k = (1 << 19) // 8 + 1, 8
    dummy = torch.zeros(8, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = lib.lib().pspec_hvp_noalloc(n, p, p, p, p, p, k, 1.5, p, None)
    assert st == lib.PSPEC_ERR_INVALID_ARG
    assert b"524288" in lib.lib().pspec_last_error()
