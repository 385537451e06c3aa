"""The host side of the row-partitioned evaluation (paper_2605_26975_gb300.shard)
on the CPU: partitions, halo sets, local renumbering, send lists built with an
all-to-all of halo requests over gloo (world size 2), the halo exchange, and
that the per-rank partial sums -- computed here by the oracle on each rank's
local graph -- add up (FP64 allreduce over gloo) to the single-rank oracle's
N, D, sigma_N, sigma_D, and the per-rank rows of Delta_p u, gradient and
Hessian product equal the whole graph's."""
import os
import socket

import numpy as np
import pytest

import oracle
from gpu_common import star_plus_powerlaw
from paper_2605_26975_gb300 import shard
from paper_2605_26975_gb300 import workloads as wl

torch = pytest.importorskip("torch")


def graphs():
    return {"grid": (wl.grid3d_longrange(2, side=8, frac_long=0.03), "block"),
            "hubs": (star_plus_powerlaw(3, n=1500), "hash")}


def owners(g, how, world):
    return shard.block_owner(g.n, world) if how == "block" else shard.hash_owner(g.n, world, seed=5)


def local_graph(plan):
    return wl.CSRGraph(plan.n_local, np.concatenate([plan.rowptr, np.full(plan.halo.size, plan.rowptr[-1])]),
                       plan.col, plan.val)


def rank_parts(plan, U, V, p):
    """What a rank's partial call computes, from the oracle on its local graph:
    N_r (1/2 the owned rows' sum), D_r, sigma_N_r, sigma_D_r and the owned
    rows of Delta_p u."""
    lg = local_graph(plan)
    Ul, Vl = plan.local_block(U), plan.local_block(V)
    no = plan.n_owned
    N = oracle.objective_parts(lg, Ul, p)[0]
    D = oracle.p_norm_p(Ul[:no], p)
    delta = oracle.p_laplacian(lg, Ul, p)[:no]
    sN = p * np.sum(delta * Vl[:no], axis=0)
    sD = p * np.sum(oracle.phi_p(Ul[:no], p) * Vl[:no], axis=0)
    return np.concatenate([N, D, sN, sD]), delta


def finish_rows(plan, U, V, p, sums, delta, k):
    """The owned rows of the gradient and the Hessian product from the added
    sums (the quotient rule of Section 2, as the finish calls apply it)."""
    N, D, sN, sD = sums[:k], sums[k:2 * k], sums[2 * k:3 * k], sums[3 * k:]
    no = plan.n_owned
    Ul, Vl = plan.local_block(U)[:no], plan.local_block(V)[:no]
    lam = N / D
    grad = (p / D) * (delta - lam * oracle.phi_p(Ul, p))
    lg = local_graph(plan)
    rows = np.repeat(np.arange(no), np.diff(plan.rowptr))
    c = p * (p - 1.0)
    Uall, Vall = plan.local_block(U), plan.local_block(V)
    S = np.zeros((no, k))
    for l in range(k):
        t = plan.val * oracle.abs_pow_pm2(Uall[rows, l] - Uall[plan.col, l], p) * (Vall[rows, l] - Vall[plan.col, l])
        S[:, l] = c * np.bincount(rows, weights=t, minlength=no)
    gN, gD = p * delta, p * oracle.phi_p(Ul, p)
    hv = (S - lam * c * oracle.abs_pow_pm2(Ul, p) * Vl) / D - (gN * sD + gD * sN - 2 * lam * gD * sD) / D ** 2
    assert lg.n == plan.n_local
    return grad, hv


def test_partitions():
    assert np.array_equal(np.bincount(shard.block_owner(10, 3)), [4, 3, 3])
    h = shard.hash_owner(1001, 4, seed=1)
    assert set(np.bincount(h)) <= {250, 251}
    assert not np.array_equal(h, shard.block_owner(1001, 4))
    o = shard.graph_owner([50, 10, 40, 30, 20], 2)
    assert np.bincount(o, weights=[50, 10, 40, 30, 20]).tolist() == [80.0, 70.0]


@pytest.mark.parametrize("name", ["grid", "hubs"])
@pytest.mark.parametrize("world", [2, 3])
def test_plans_and_sums_single_process(name, world):
    g, how = graphs()[name]
    owner = owners(g, how, world)
    plans = [shard.ShardPlan.build(g, owner, r, world) for r in range(world)]
    # every vertex owned once; local CSR = the global rows; halo = foreign neighbours
    assert np.array_equal(np.sort(np.concatenate([pl.owned for pl in plans])), np.arange(g.n))
    for pl in plans:
        ids = pl.local_ids
        for t, i in enumerate(pl.owned[:50]):
            glob = g.col[g.rowptr[i]:g.rowptr[i + 1]]
            assert np.array_equal(ids[pl.col[pl.rowptr[t]:pl.rowptr[t + 1]]], glob)
        nb = np.unique(np.concatenate([g.col[g.rowptr[i]:g.rowptr[i + 1]] for i in pl.owned]))
        assert np.array_equal(np.sort(pl.halo), nb[owner[nb] != pl.rank])
        # what rank q sends this rank is exactly this rank's halo slice owned by q
        offs = np.concatenate([[0], np.cumsum(pl.halo_counts)])
        for q in range(world):
            got = plans[q].owned[plans[q].send[pl.rank]]
            assert np.array_equal(got, pl.halo[offs[q]:offs[q + 1]])
    k, p = 3, 1.4
    U = wl.orthonormal_block(7, g.n, k).astype(np.float64)
    V = wl.gaussian_block(8, g.n, k).astype(np.float64)
    parts = [rank_parts(pl, U, V, p) for pl in plans]
    sums = np.sum([s for s, _ in parts], axis=0)
    N, D = oracle.objective_parts(g, U, p)
    delta_ref = oracle.p_laplacian(g, U, p)
    assert np.allclose(sums[:k], N, rtol=1e-12, atol=0) and np.allclose(sums[k:2 * k], D, rtol=1e-13, atol=0)
    assert np.allclose(sums[2 * k:3 * k], p * np.sum(delta_ref * V, 0), rtol=1e-10, atol=1e-12)
    assert np.allclose(sums[3 * k:], p * np.sum(oracle.phi_p(U, p) * V, 0), rtol=1e-12, atol=1e-14)
    g_ref, h_ref = oracle.euclidean_grad(g, U, p), oracle.euclidean_hvp(g, U, V, p)
    for pl, (_, delta) in zip(plans, parts):
        assert np.allclose(delta, delta_ref[pl.owned], rtol=1e-13, atol=1e-15)
        gr, hv = finish_rows(pl, U, V, p, sums, delta, k)
        assert np.allclose(gr, g_ref[pl.owned], rtol=1e-10, atol=1e-13)
        assert np.allclose(hv, h_ref[pl.owned], rtol=1e-10, atol=1e-13)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, how = graphs()[name]
        owner = owners(g, how, world)
        plan = shard.ShardPlan.build(g, owner, rank, world, dist=dist)
        ref = shard.ShardPlan.build(g, owner, rank, world)
        same_send = all(np.array_equal(a, b) for a, b in zip(plan.send, ref.send))
        k, p = 4, 1.3
        U = wl.orthonormal_block(7, g.n, k).astype(np.float64)
        V = wl.gaussian_block(8, g.n, k).astype(np.float64)
        # the halo rows arrive through the exchange only: start from garbage
        Ul = torch.from_numpy(plan.local_block(U))
        Vl = torch.from_numpy(plan.local_block(V))
        Ul[plan.n_owned:] = float("nan")
        Vl[plan.n_owned:] = float("nan")
        plan.exchange(Ul, dist)
        plan.exchange(Vl, dist)
        halo_ok = bool(torch.equal(Ul, torch.from_numpy(plan.local_block(U))) and
                       torch.equal(Vl, torch.from_numpy(plan.local_block(V))))
        sums, delta = rank_parts(plan, U, V, p)
        t = torch.from_numpy(sums.copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        gr, hv = finish_rows(plan, U, V, p, t.numpy(), delta, k)
        out[rank] = (same_send, halo_ok, t.numpy(), plan.owned, gr, hv)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["grid", "hubs"])
def test_two_ranks_over_gloo(name):
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), name, out), nprocs=world, join=True)
        res = dict(out)
    g, _ = graphs()[name]
    k, p = 4, 1.3
    U = wl.orthonormal_block(7, g.n, k).astype(np.float64)
    V = wl.gaussian_block(8, g.n, k).astype(np.float64)
    N, D = oracle.objective_parts(g, U, p)
    g_ref, h_ref = oracle.euclidean_grad(g, U, p), oracle.euclidean_hvp(g, U, V, p)
    for r in range(world):
        same_send, halo_ok, sums, owned, gr, hv = res[r]
        assert same_send and halo_ok
        assert np.allclose(sums[:k], N, rtol=1e-12, atol=0) and np.allclose(sums[k:2 * k], D, rtol=1e-13, atol=0)
        assert np.allclose(gr, g_ref[owned], rtol=1e-10, atol=1e-13)
        assert np.allclose(hv, h_ref[owned], rtol=1e-10, atol=1e-13)
    assert np.array_equal(res[0][2], res[1][2])  # every rank holds the same added sums
