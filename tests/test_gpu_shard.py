"""The row-partitioned calls of the C ABI (pspec_graph_create_shard,
pspec_*_partial, pspec_*_finish) on one GPU.  Several ranks are emulated as
independent calls in sequence -- each shard its own handle and block, the
FP64 allreduce done by adding the ranks' sums -- so nothing on the GPU waits
for another rank.  The assembled objective, gradient and Hessian product
match the FP64 oracle on the whole graph and the whole-graph handle.  A
one-rank ShardedGraph over gloo checks the Python driver end to end."""
import numpy as np
import pytest

import oracle
from gpu_common import (TOL_F, TOL_GRAD, TOL_HVP, grad_term_scale, rel_col, rel_elem,
                        star_plus_powerlaw)
from paper_2605_26975_gb300 import shard
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


def graph(name):
    return {"hubs": lambda: star_plus_powerlaw(3, n=6000),
            "grid": lambda: wl.grid3d_longrange(2, side=14, frac_long=0.01),
            "knn": lambda: wl.knn_gaussian_mixture(5, n=5000, mixtures=4)}[name]()


CASES = [("hubs", "hash", 8, 3), ("grid", "block", 8, 2), ("hubs", "block", 16, 4), ("knn", "hash", 4, 3),
         ("grid", "hash", 3, 2)]


@pytest.mark.parametrize("name,how,k,world", CASES, ids=[f"{c[0]}-{c[1]}-k{c[2]}-w{c[3]}" for c in CASES])
def test_emulated_ranks_match_oracle(api, name, how, k, world):
    g = graph(name)
    owner = shard.block_owner(g.n, world) if how == "block" else shard.hash_owner(g.n, world, seed=2)
    plans = [shard.ShardPlan.build(g, owner, r, world) for r in range(world)]
    shards = [api.Shard(pl.n_owned, pl.n_local, pl.rowptr, pl.col, pl.val) for pl in plans]
    U = wl.orthonormal_block(11, g.n, k, np.float32)
    V = wl.gaussian_block(12, g.n, k, dtype=np.float32)
    U64, V64 = U.astype(np.float64), V.astype(np.float64)
    whole = api.Graph.from_csr(g)
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    for p in (1.3, 2.0, 1.1):
        Uls = [torch.from_numpy(pl.local_block(U)).cuda() for pl in plans]
        Vls = [torch.from_numpy(pl.local_block(V)).cuda() for pl in plans]
        # objective and gradient: partial sums, added over the ranks, finish
        outs = [S.eval_partial(Ul, p) for S, Ul in zip(shards, Uls)]
        total = torch.stack([s for _, s in outs]).sum(0)
        grad = np.zeros((g.n, k))
        Fs = []
        for pl, S, Ul, (gr, _) in zip(plans, shards, Uls, outs):
            F, gr = S.eval_finish(Ul, p, total, gr)
            Fs.append(F.item())
            grad[pl.owned] = gr[:pl.n_owned].cpu().numpy()
        # Hessian product
        houts = [S.hvp_partial(Ul, Vl, p) for S, Ul, Vl in zip(shards, Uls, Vls)]
        htotal = torch.stack([s for _, s in houts]).sum(0)
        hv = np.zeros((g.n, k))
        for pl, S, Ul, Vl, (h, _) in zip(plans, shards, Uls, Vls, houts):
            hv[pl.owned] = S.hvp_finish(Ul, Vl, p, htotal, h)[:pl.n_owned].cpu().numpy()
        torch.cuda.synchronize()
        for S in shards:
            assert S.status() == 0
        F_ref = oracle.objective(g, U64, p)
        assert max(abs(F - F_ref) for F in Fs) <= TOL_F * F_ref
        g_ref = oracle.euclidean_grad(g, U64, p)
        assert rel_col(grad, g_ref) <= TOL_GRAD
        assert rel_elem(grad, g_ref, grad_term_scale(oracle, g, U64, p)) <= TOL_GRAD
        assert rel_col(hv, oracle.euclidean_hvp(g, U64, V64, p)) <= TOL_HVP
        # and the whole-graph handle within rounding of the summation order
        _, gw = whole.eval(Ud, p)
        hw = whole.hvp(Ud, Vd, p)
        assert rel_col(grad, gw.cpu().numpy().astype(np.float64)) <= TOL_GRAD
        assert rel_col(hv, hw.cpu().numpy().astype(np.float64)) <= TOL_HVP


def test_shard_rejects_whole_graph_calls(api):
    from paper_2605_26975_gb300 import _abi
    g = graph("grid")
    pl = shard.ShardPlan.build(g, shard.block_owner(g.n, 2), 0, 2)
    S = api.Shard(pl.n_owned, pl.n_local, pl.rowptr, pl.col, pl.val)
    U = torch.from_numpy(pl.local_block(wl.orthonormal_block(1, g.n, 4, np.float32))).cuda()
    out = torch.empty_like(U)
    import ctypes as C
    st = _abi.lib().pspec_eval(S.handle, C.c_void_p(U.data_ptr()), 4, 1.5, _abi.PSPEC_F32, None,
                               C.c_void_p(out.data_ptr()), None, 0, None)
    assert st == _abi.PSPEC_ERR_INVALID_ARG
    sums = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(_abi.PspecError):
        S.hvp_finish(U, U.clone(), 1.5, sums, out)  # no partial call before it
    with pytest.raises(TypeError):
        S.eval_partial(U.double(), 1.5)  # the binding refuses FP64 before the library would


def test_sharded_graph_one_rank_over_gloo(api, tmp_path):
    """ShardedGraph with one rank (no halo): the exchange, the partial calls,
    the allreduce through torch.distributed and the finish calls give the
    whole-graph handle's results."""
    import torch.distributed as dist
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    dist.init_process_group("gloo", init_method=f"file://{tmp_path}/pg", rank=0, world_size=1)
    try:
        g = graph("hubs")
        plan = shard.ShardPlan.build(g, np.zeros(g.n, dtype=np.int32), 0, 1, dist=dist)
        SG = shard.ShardedGraph(plan, dist)
        U = wl.orthonormal_block(3, g.n, 8, np.float32)
        V = wl.gaussian_block(4, g.n, 8, dtype=np.float32)
        Ul, Vl = torch.from_numpy(plan.local_block(U)).cuda(), torch.from_numpy(plan.local_block(V)).cuda()
        F, gr = SG.eval(Ul, 1.3)
        hv = SG.hvp(Ul, Vl, 1.3)
        whole = api.Graph.from_csr(g)
        Fw, gw = whole.eval(torch.from_numpy(U).cuda(), 1.3)
        hw = whole.hvp(torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), 1.3)
        torch.cuda.synchronize()
        assert abs(F.item() - Fw.item()) <= 1e-12 * Fw.item()
        inv = np.argsort(plan.local_ids)
        assert torch.equal(gr.cpu()[inv], gw.cpu()) and torch.equal(hv.cpu()[inv], hw.cpu())
    finally:
        dist.destroy_process_group()
