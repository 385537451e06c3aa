"""Row-partitioned evaluation over several GPUs: the host side.

Every per-column quantity of the method (Section 2: N_l, D_l and the Hessian
product's sigma_N, sigma_D) is a sum over the rows of W, so the rows can be
split over ranks (one process and one GPU each): a rank owns a set of
vertices, evaluates the rows of its owned vertices, and needs U (and V) on
the neighbours of those rows that other ranks own -- its halo.  One Newton
step's evaluation is then

    halo exchange of U (and V)  ->  per-rank partial sums (the library's
    pspec_*_partial calls)  ->  FP64 allreduce of 2k or 4k sums  ->
    per-rank epilogue on the owned rows (pspec_*_finish),

the only collective being the allreduce of the O(k) sums and the halo rows
themselves (copied into local memory before the kernels run; no kernel reads
another GPU's memory).  Graph batches shard by graph instead and need no
exchange at all (`graph_owner`).

This module builds the partition (`block_owner`, `hash_owner`), each rank's
plan (`ShardPlan.build`: owned vertices, the halo sorted by owner, the local
CSR with columns renumbered owned-first then halo, and the send lists, set up
with one all-to-all of halo requests), the exchange (`ShardPlan.exchange`),
and `ShardedGraph`, which runs the steps above through the C ABI.  The
exchange and the reductions go through torch.distributed, so the same code
runs on gloo (CPU tensors; the tests) and NCCL (CUDA tensors).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def block_owner(n: int, world: int) -> np.ndarray:
    """Contiguous blocks of rows: vertex i belongs to rank floor(i * world / n)
    (the natural split of a grid in its own order)."""
    return (np.arange(n, dtype=np.int64) * world // n).astype(np.int32)


def hash_owner(n: int, world: int, seed: int = 0) -> np.ndarray:
    """A balanced pseudo-random split for graphs without a useful order: a
    seeded permutation of the vertices dealt out in blocks."""
    perm = np.random.default_rng(seed).permutation(n)
    owner = np.empty(n, dtype=np.int32)
    owner[perm] = block_owner(n, world)
    return owner


def graph_owner(sizes, world: int) -> np.ndarray:
    """Graphs of a batch to ranks, largest first onto the least loaded rank
    (no exchange: a graph's rows never leave its rank)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(sizes.size, dtype=np.int32)
    for g in np.argsort(-sizes, kind="stable"):
        r = int(np.argmin(load))
        owner[g] = r
        load[r] += sizes[g]
    return owner


@dataclasses.dataclass
class ShardPlan:
    rank: int
    world: int
    owned: np.ndarray        # int64 global ids of the owned vertices, ascending
    halo: np.ndarray         # int64 global ids of the halo, sorted by (owner, id)
    halo_counts: np.ndarray  # halo vertices owned by each rank (0 for this rank)
    send: list               # per rank: local indices of owned rows it needs, in its halo order
    rowptr: np.ndarray       # local CSR of the owned rows (n_owned + 1)
    col: np.ndarray          # int32 local columns: owned 0..n_owned-1, halo after
    val: np.ndarray

    @property
    def n_owned(self) -> int:
        return int(self.owned.size)

    @property
    def n_local(self) -> int:
        return int(self.owned.size + self.halo.size)

    @property
    def local_ids(self) -> np.ndarray:
        """Global id of every local vertex (owned, then halo)."""
        return np.concatenate([self.owned, self.halo])

    @classmethod
    def build(cls, g, owner: np.ndarray, rank: int, world: int, dist=None, group=None) -> "ShardPlan":
        """This rank's plan from the global CSR g and the owner of every vertex.
        The send lists come from one all-to-all of halo requests when a
        process group is given (each rank then needs only its own rows of g);
        without one (a single process emulating every rank) they are worked
        out from the global graph."""
        owner = np.asarray(owner, dtype=np.int32)
        owned = np.flatnonzero(owner == rank).astype(np.int64)
        rp = np.asarray(g.rowptr, dtype=np.int64)
        idx, lens = _row_entries(rp, owned)
        gcol = np.asarray(g.col, dtype=np.int64)[idx]
        val = np.asarray(g.val)[idx]
        nb = np.unique(gcol)
        nb = nb[owner[nb] != rank]
        order = np.lexsort((nb, owner[nb]))
        halo = nb[order]
        halo_counts = np.bincount(owner[halo], minlength=world).astype(np.int64)
        local = np.full(g.n, -1, dtype=np.int64)
        local[owned] = np.arange(owned.size)
        local[halo] = owned.size + np.arange(halo.size)
        col = local[gcol].astype(np.int32)
        rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        plan = cls(rank, world, owned, halo, halo_counts, [], rowptr, col, val)
        if dist is not None:
            requests = plan._exchange_requests(dist, group)
        else:
            requests = []
            for q in range(world):
                hq = cls._halo_of(g, owner, q) if q != rank else np.zeros(0, dtype=np.int64)
                requests.append(hq[owner[hq] == rank])
        plan.send = [local[np.asarray(r, dtype=np.int64)] for r in requests]
        assert all(np.all(s >= 0) and np.all(s < owned.size) for s in plan.send)
        return plan

    @staticmethod
    def _halo_of(g, owner, q):
        rp = np.asarray(g.rowptr, dtype=np.int64)
        idx, _ = _row_entries(rp, np.flatnonzero(owner == q))
        nb = np.unique(np.asarray(g.col, dtype=np.int64)[idx])
        nb = nb[owner[nb] != q]
        return nb[np.lexsort((nb, owner[nb]))]

    def _exchange_requests(self, dist, group):
        """Tell every owner which of its vertices this rank's halo holds;
        returns, per rank, the global ids it asked this rank for."""
        import torch
        dev = _device_of(dist, group)
        counts_out = torch.tensor(self.halo_counts, dtype=torch.int64, device=dev)
        counts_in = torch.empty_like(counts_out)
        dist.all_to_all_single(counts_in, counts_out, group=group)
        cin = counts_in.cpu().numpy()
        ids_in = torch.empty(int(cin.sum()), dtype=torch.int64, device=dev)
        dist.all_to_all_single(ids_in, torch.as_tensor(self.halo, device=dev),
                               output_split_sizes=cin.tolist(),
                               input_split_sizes=self.halo_counts.tolist(), group=group)
        ids = ids_in.cpu().numpy()
        offs = np.concatenate([[0], np.cumsum(cin)])
        return [ids[offs[q]:offs[q + 1]] for q in range(self.world)]

    def exchange(self, X, dist, group=None):
        """Fill the halo rows X[n_owned:] (X: n_local x k tensor on the
        group's device) with their owners' values: one all-to-all of rows."""
        import torch
        if self.world == 1:
            return X  # a single rank has no halo
        send_idx = torch.as_tensor(np.concatenate(self.send).astype(np.int64), device=X.device)
        out = torch.empty((self.halo.size,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
        dist.all_to_all_single(out, X.index_select(0, send_idx).contiguous(),
                               output_split_sizes=self.halo_counts.tolist(),
                               input_split_sizes=[int(s.size) for s in self.send], group=group)
        X[self.n_owned:] = out
        return X

    def local_block(self, X_global):
        """The rows of a global n x k array this rank holds (owned, then halo)."""
        return np.ascontiguousarray(np.asarray(X_global)[self.local_ids])


def _row_entries(rp, rows):
    """Positions of the stored entries of the given rows (in row order) and
    the rows' lengths."""
    lens = rp[rows + 1] - rp[rows]
    first = np.repeat(rp[rows] - (np.cumsum(lens) - lens), lens)
    return first + np.arange(int(lens.sum()), dtype=np.int64), lens


def _device_of(dist, group):
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


class ShardedGraph:
    """One rank's share of W on its GPU: F, gradient and Hessian product of the
    whole graph, restricted to the owned rows, through the library's
    row-partitioned calls (halo exchange, partial sums, FP64 allreduce,
    finish)."""

    def __init__(self, plan: ShardPlan, dist, group=None):
        from . import api
        self.plan, self.dist, self.group = plan, dist, group
        self.G = api.Shard(plan.n_owned, plan.n_local, plan.rowptr, plan.col, plan.val)

    def _allreduce(self, sums):
        if sums.is_cuda and _device_of(self.dist, self.group) == "cpu":  # gloo: through the host
            host = sums.cpu()
            self.dist.all_reduce(host, op=self.dist.ReduceOp.SUM, group=self.group)
            return sums.copy_(host)
        self.dist.all_reduce(sums, op=self.dist.ReduceOp.SUM, group=self.group)
        return sums

    def eval(self, U_local, p, exchange=True):
        """(F, gradient on the owned rows); U_local is n_local x k FP32 on this
        rank's GPU, its halo rows refreshed here unless exchange=False."""
        if exchange:
            self.plan.exchange(U_local, self.dist, self.group)
        grad, sums = self.G.eval_partial(U_local, p)
        F, grad = self.G.eval_finish(U_local, p, self._allreduce(sums), grad)
        return F, grad

    def hvp(self, U_local, V_local, p, exchange=True):
        """The exact Hessian product on the owned rows (halo rows of U and V
        refreshed unless exchange=False)."""
        if exchange:
            self.plan.exchange(U_local, self.dist, self.group)
            self.plan.exchange(V_local, self.dist, self.group)
        HV, sums = self.G.hvp_partial(U_local, V_local, p)
        return self.G.hvp_finish(U_local, V_local, p, self._allreduce(sums), HV)
