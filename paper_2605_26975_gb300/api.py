"""Python binding of the C ABI on torch tensors (marshalling only).

Every computation runs in libpspec.so's CUDA kernels; this module only checks
tensor placement and dtypes, passes data pointers and the current CUDA
stream, and raises PspecError on a non-OK status.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import check, lib

_DT = {torch.float32: _abi.PSPEC_F32, torch.float64: _abi.PSPEC_F64}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev_block(t, name, n=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in _DT:
        raise TypeError(f"{name} must be float32 or float64")
    if t.dim() != 2 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous n x k tensor")
    if n is not None and t.shape[0] != n:
        raise ValueError(f"{name} has {t.shape[0]} rows, the graph has {n}")
    return t


class Graph:
    """A symmetric weight matrix W on the device (pspec_graph_create)."""

    def __init__(self, rowptr, col, val, check_symmetry=False, node_off=None):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val)
        if val.dtype not in (np.float32, np.float64):
            val = val.astype(np.float64)
        vt = _abi.PSPEC_F32 if val.dtype == np.float32 else _abi.PSPEC_F64
        flags = _abi.PSPEC_HOST_PTRS | (_abi.PSPEC_CHECK_SYMMETRY if check_symmetry else 0)
        h = C.c_void_p()
        if node_off is None:
            st = lib().pspec_graph_create(rowptr.size - 1, rowptr.ctypes.data, col.ctypes.data,
                                          val.ctypes.data, vt, flags, _stream(), C.byref(h))
            check(st, "pspec_graph_create")
        else:
            node_off = np.ascontiguousarray(node_off, dtype=np.int64)
            st = lib().pspec_graph_create_batched(node_off.size - 1, node_off.ctypes.data,
                                                  rowptr.ctypes.data, col.ctypes.data,
                                                  val.ctypes.data, vt, flags, _stream(), C.byref(h))
            check(st, "pspec_graph_create_batched")
        self._h = h
        n, nnz, ng = C.c_int64(), C.c_int64(), C.c_int32()
        check(lib().pspec_graph_info(h, C.byref(n), C.byref(nnz), C.byref(ng)), "pspec_graph_info")
        self.n, self.nnz, self.n_graphs = n.value, nnz.value, ng.value

    @classmethod
    def from_csr(cls, g, **kw):
        return cls(g.rowptr, g.col, g.val, **kw)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib().pspec_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ per call
    def eval(self, U, p, grad_out=None, parts=False, keep_delta=False):
        """(F, grad[, parts]): F a float64 CUDA tensor with one entry per graph
        of the handle, parts [n_graphs * 2k] (each graph's N_1..N_k, D_1..D_k).
        keep_delta=True keeps Delta_p u on the handle for hvp(..., delta_kept=True)
        at the same U (FP32, single graph)."""
        U = _dev_block(U, "U", self.n)
        k = U.shape[1]
        G = self.n_graphs
        grad = torch.empty_like(U) if grad_out is None else grad_out
        F = torch.empty(G, dtype=torch.float64, device=U.device)
        P = torch.empty(G * 2 * k, dtype=torch.float64, device=U.device) if parts else None
        flags = _abi.PSPEC_KEEP_DELTA if keep_delta else 0
        st = lib().pspec_eval(self._h, _ptr(U), k, float(p), _DT[U.dtype], _ptr(F), _ptr(grad),
                              _ptr(P), flags, _stream())
        check(st, "pspec_eval")
        return (F, grad, P) if parts else (F, grad)

    def hvp(self, U, V, p, out=None, alg1=False, delta_kept=False):
        """Exact Hessian of F_p at U applied to V; alg1=True leaves out the
        rank-two terms (the sparse-plus-diagonal form of Algorithm 1);
        delta_kept=True reuses the Delta_p u kept by eval(U, p, keep_delta=True)
        (same tensor U, unchanged since)."""
        U = _dev_block(U, "U", self.n)
        V = _dev_block(V, "V", self.n)
        if V.shape != U.shape or V.dtype != U.dtype:
            raise ValueError("U and V must have the same shape and dtype")
        HV = torch.empty_like(U) if out is None else out
        flags = (_abi.PSPEC_HVP_ALG1 if alg1 else 0) | (_abi.PSPEC_DELTA_KEPT if delta_kept else 0)
        st = lib().pspec_hvp(self._h, _ptr(U), _ptr(V), U.shape[1], float(p), _DT[U.dtype],
                             _ptr(HV), flags, _stream())
        check(st, "pspec_hvp")
        return HV

    def eval_host(self, U, p, grad_out, keep_delta=False):
        """pspec_eval with PSPEC_HOST_PTRS: U and grad_out are CPU tensors
        (pinned for asynchronous copies); returns F as a Python float (a list
        of floats, one per graph, for a batched handle)."""
        k = U.shape[1]
        F = (C.c_double * self.n_graphs)()
        flags = _abi.PSPEC_HOST_PTRS | (_abi.PSPEC_KEEP_DELTA if keep_delta else 0)
        st = lib().pspec_eval(self._h, C.c_void_p(U.data_ptr()), k, float(p), _DT[U.dtype],
                              F, C.c_void_p(grad_out.data_ptr()), None, flags, _stream())
        check(st, "pspec_eval(host)")
        return F[0] if self.n_graphs == 1 else list(F)

    def hvp_host(self, U, V, p, out, delta_kept=False):
        flags = _abi.PSPEC_HOST_PTRS | (_abi.PSPEC_DELTA_KEPT if delta_kept else 0)
        st = lib().pspec_hvp(self._h, C.c_void_p(U.data_ptr()), C.c_void_p(V.data_ptr()),
                             U.shape[1], float(p), _DT[U.dtype], C.c_void_p(out.data_ptr()),
                             flags, _stream())
        check(st, "pspec_hvp(host)")
        return out

    def tune(self, U, V, p, reps=5):
        """pspec_tune: time the edge kernels' launch shapes on U, V (FP32 CUDA
        tensors) and keep the fastest on this handle.  Returns the candidates
        [(edges_per_lane, blocks_per_sm, ms)] and the chosen index."""
        U = _dev_block(U, "U", self.n)
        V = _dev_block(V, "V", self.n)
        if U.dtype != torch.float32 or V.dtype != torch.float32 or V.shape != U.shape:
            raise TypeError("U and V must be float32 tensors of the same shape")
        rep = _abi.TuneReport()
        check(lib().pspec_tune(self._h, _ptr(U), _ptr(V), U.shape[1], float(p), int(reps),
                               C.byref(rep), _stream()), "pspec_tune")
        cands = [(rep.edges_per_lane[i], rep.blocks_per_sm[i], rep.ms[i]) for i in range(rep.n_candidates)]
        return cands, rep.chosen

    def status(self):
        """Synchronise and return (and clear) the kernel-recorded status."""
        return lib().pspec_graph_status(self._h, _stream())

    # --------------------------------------------------------------- solve
    def solve(self, U0, p_schedule, opts=None, labels=True):
        """Trust-region Newton + tCG over the p schedule, k-means, RCut.
        Returns (U, labels, rcut, stats dict, status)."""
        U = _dev_block(U0, "U0", self.n).clone()
        k = U.shape[1]
        o = default_opts() if opts is None else opts
        sched = np.ascontiguousarray(p_schedule, dtype=np.float64)
        lab = torch.empty(self.n, dtype=torch.int32, device=U.device) if labels else None
        rc = C.c_double(float("nan"))
        stats = _abi.SolveStats()
        st = lib().pspec_solve(self._h, k, sched.ctypes.data, sched.size, C.byref(o), _DT[U.dtype],
                               _ptr(U), _ptr(lab), C.byref(rc), C.byref(stats), _stream())
        check(st, "pspec_solve", allow=(_abi.PSPEC_OK, _abi.PSPEC_ERR_NOT_CONVERGED))
        ns = stats.n_stages
        sd = dict(outer=list(stats.outer[:ns]), inner=list(stats.inner[:ns]), f=list(stats.f[:ns]),
                  gnorm=list(stats.gnorm[:ns]), hvp_calls=stats.hvp_calls,
                  eval_calls=stats.eval_calls, seconds=stats.seconds,
                  kmeans_inertia=stats.kmeans_inertia)
        return U, lab, rc.value, sd, st

    def solve_batched(self, U0, p_schedule, opts=None, threads=16):
        """pspec_solve_batched on a batched handle: every graph solved on its
        own, concurrently.  U0 is the concatenated n x k FP32 block.  Returns
        (U, labels (per-graph 0..k-1), rcut per graph, status per graph,
        overall status)."""
        if self.n_graphs < 1:
            raise ValueError("not a graph handle")
        U = _dev_block(U0, "U0", self.n).clone()
        if U.dtype != torch.float32:
            raise TypeError("the batched solve runs the FP32 path")
        k = U.shape[1]
        o = default_opts() if opts is None else opts
        sched = np.ascontiguousarray(p_schedule, dtype=np.float64)
        lab = torch.empty(self.n, dtype=torch.int32, device=U.device)
        rc = np.zeros(self.n_graphs, dtype=np.float64)
        status = np.zeros(self.n_graphs, dtype=np.int32)
        st = lib().pspec_solve_batched(self._h, k, sched.ctypes.data, sched.size, C.byref(o), _ptr(U),
                                       _ptr(lab), rc.ctypes.data, status.ctypes.data, int(threads),
                                       _stream())
        check(st, "pspec_solve_batched", allow=(_abi.PSPEC_OK, _abi.PSPEC_ERR_NOT_CONVERGED))
        return U, lab, rc, status, st

    def solve_lockstep(self, U0, p_schedule, opts=None, threads=16, allow_errors=False):
        """pspec_solve_lockstep on a batched handle: every graph's solve with
        the whole batch stepping together on the device.  Returns (U, labels,
        rcut per graph, status per graph, stats per graph (dicts), overall
        status).  With allow_errors a per-graph error does not raise."""
        if self.n_graphs < 1:
            raise ValueError("not a graph handle")
        U = _dev_block(U0, "U0", self.n).clone()
        if U.dtype != torch.float32:
            raise TypeError("the lockstep solve runs the FP32 path")
        k = U.shape[1]
        o = default_opts() if opts is None else opts
        sched = np.ascontiguousarray(p_schedule, dtype=np.float64)
        lab = torch.zeros(self.n, dtype=torch.int32, device=U.device)
        G = self.n_graphs
        rc = np.zeros(G, dtype=np.float64)
        status = np.zeros(G, dtype=np.int32)
        stats = (_abi.SolveStats * G)()
        st = lib().pspec_solve_lockstep(self._h, k, sched.ctypes.data, sched.size, C.byref(o), _ptr(U),
                                        _ptr(lab), rc.ctypes.data, status.ctypes.data, stats, int(threads),
                                        _stream())
        if not allow_errors:
            check(st, "pspec_solve_lockstep", allow=(_abi.PSPEC_OK, _abi.PSPEC_ERR_NOT_CONVERGED))
        ns = sched.size
        sd = [dict(outer=list(x.outer[:ns]), inner=list(x.inner[:ns]), f=list(x.f[:ns]),
                   gnorm=list(x.gnorm[:ns]), hvp_calls=x.hvp_calls, eval_calls=x.eval_calls,
                   seconds=x.seconds, kmeans_inertia=x.kmeans_inertia) for x in stats]
        return U, lab, rc, status, sd, st

    def rcut(self, labels, n_clusters):
        if not labels.is_cuda or labels.dtype != torch.int32:
            raise TypeError("labels must be an int32 CUDA tensor")
        out = C.c_double()
        check(lib().pspec_rcut(self._h, _ptr(labels), int(n_clusters), C.byref(out), _stream()),
              "pspec_rcut")
        return out.value

    # --------------------------------------------------------- timing
    def set_timing(self, enable=True):
        check(lib().pspec_set_timing(self._h, 1 if enable else 0), "pspec_set_timing")

    def kernel_times(self):
        """{kernel name: (launches, total ms)} since the last call."""
        buf = C.create_string_buffer(8192)
        check(lib().pspec_kernel_times(self._h, buf, len(buf)), "pspec_kernel_times")
        out = {}
        for item in buf.value.decode().split(";"):
            if item:
                name, rest = item.split("=")
                cnt, ms = rest.split(":")
                out[name] = (int(cnt), float(ms))
        return out


class Shard:
    """One rank's rows of a row-partitioned W (pspec_graph_create_shard): the
    owned rows' CSR with local columns (owned vertices first, halo after).
    Its calls return partial FP64 sums for the caller to add over ranks, and
    finish the owned rows from the added sums."""

    def __init__(self, n_owned, n_local, rowptr, col, val):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val)
        if val.dtype not in (np.float32, np.float64):
            val = val.astype(np.float64)
        vt = _abi.PSPEC_F32 if val.dtype == np.float32 else _abi.PSPEC_F64
        h = C.c_void_p()
        check(lib().pspec_graph_create_shard(int(n_owned), int(n_local), rowptr.ctypes.data, col.ctypes.data,
                                             val.ctypes.data, vt, _abi.PSPEC_HOST_PTRS, _stream(),
                                             C.byref(h)), "pspec_graph_create_shard")
        self._h = h
        self.n_owned, self.n_local = int(n_owned), int(n_local)

    close = Graph.close
    __del__ = Graph.__del__
    status = Graph.status

    @property
    def handle(self):
        return self._h

    def _blocks(self, *ts):
        for t in ts:
            _dev_block(t, "block", self.n_local)
            if t.dtype != torch.float32:
                raise TypeError("the row-partitioned calls run the FP32 path")

    def eval_partial(self, U, p, grad_out=None):
        """(Delta_p u rows in grad_out, FP64 sums [N_r, D_r]) of the owned rows."""
        self._blocks(U)
        k = U.shape[1]
        grad = torch.empty_like(U) if grad_out is None else grad_out
        sums = torch.empty(2 * k, dtype=torch.float64, device=U.device)
        check(lib().pspec_eval_partial(self._h, _ptr(U), k, float(p), _ptr(grad), _ptr(sums), _stream()),
              "pspec_eval_partial")
        return grad, sums

    def eval_finish(self, U, p, sums, grad):
        """(F, gradient of the owned rows) from the sums added over ranks."""
        k = U.shape[1]
        F = torch.empty(1, dtype=torch.float64, device=U.device)
        check(lib().pspec_eval_finish(self._h, _ptr(U), k, float(p), _ptr(sums), _ptr(F), _ptr(grad),
                                      _stream()), "pspec_eval_finish")
        return F, grad

    def hvp_partial(self, U, V, p, out=None):
        """(sparse part of the owned rows in out, FP64 sums [N_r, D_r, sigma_N_r, sigma_D_r])."""
        self._blocks(U, V)
        k = U.shape[1]
        HV = torch.empty_like(U) if out is None else out
        sums = torch.empty(4 * k, dtype=torch.float64, device=U.device)
        check(lib().pspec_hvp_partial(self._h, _ptr(U), _ptr(V), k, float(p), _ptr(HV), _ptr(sums),
                                      _stream()), "pspec_hvp_partial")
        return HV, sums

    def hvp_finish(self, U, V, p, sums, HV, alg1=False):
        """The Hessian product of the owned rows from the sums added over ranks."""
        check(lib().pspec_hvp_finish(self._h, _ptr(U), _ptr(V), U.shape[1], float(p), _ptr(sums), _ptr(HV),
                                     _abi.PSPEC_HVP_ALG1 if alg1 else 0, _stream()), "pspec_hvp_finish")
        return HV


def default_opts(**kw):
    o = _abi.SolveOpts()
    lib().pspec_solve_opts_default(C.byref(o))
    for key, v in kw.items():
        setattr(o, key, v)
    return o


def kmeans(X, n_clusters, seed=0, restarts=10, max_iter=300):
    """k-means of the rows of X (CUDA tensor); returns (labels, centers, inertia)."""
    X = _dev_block(X, "X")
    n, dim = X.shape
    labels = torch.empty(n, dtype=torch.int32, device=X.device)
    centers = torch.empty((n_clusters, dim), dtype=torch.float64, device=X.device)
    inertia = C.c_double()
    st = lib().pspec_kmeans(_ptr(X), n, dim, _DT[X.dtype], int(n_clusters), C.c_uint64(seed),
                            int(restarts), int(max_iter), _ptr(labels), _ptr(centers),
                            C.byref(inertia), _stream())
    check(st, "pspec_kmeans")
    return labels, centers, inertia.value


def version():
    return lib().pspec_version().decode()
