"""ctypes declarations of the C ABI in include/pspec.h (argument marshalling only).

The library is the in-tree libpspec.so built by ``paper_2605_26975_gb300.build``.
Loading fails loudly when it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpspec.so")

PSPEC_OK = 0
PSPEC_ERR_INVALID_ARG = 1
PSPEC_ERR_CUDA = 2
PSPEC_ERR_OOM = 3
PSPEC_ERR_ZERO_COLUMN = 4
PSPEC_ERR_NONFINITE = 5
PSPEC_ERR_NOT_CONVERGED = 6
PSPEC_ERR_TIMEOUT = 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "ZERO_COLUMN",
                5: "NONFINITE", 6: "NOT_CONVERGED", 7: "TIMEOUT"}

PSPEC_F32 = 0
PSPEC_F64 = 1
PSPEC_HOST_PTRS = 0x1
PSPEC_CHECK_SYMMETRY = 0x2
PSPEC_HVP_ALG1 = 0x4
PSPEC_KEEP_DELTA = 0x8
PSPEC_DELTA_KEPT = 0x10
PSPEC_HESSIAN_EXACT = 0
PSPEC_HESSIAN_ALG1 = 1


class SolveOpts(C.Structure):
    _fields_ = [("max_outer", C.c_int32), ("max_inner", C.c_int32), ("gtol_rel", C.c_double),
                ("gtol_abs", C.c_double), ("theta", C.c_double), ("kappa", C.c_double),
                ("delta_bar_scale", C.c_double), ("delta0_scale", C.c_double),
                ("rho_prime", C.c_double), ("rho_reg", C.c_double),
                ("kmeans_restarts", C.c_int32), ("kmeans_max_iter", C.c_int32),
                ("seed", C.c_uint64), ("verbose", C.c_int32), ("hessian_form", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("n_stages", C.c_int32), ("outer", C.c_int32 * 32), ("inner", C.c_int32 * 32),
                ("f", C.c_double * 32), ("gnorm", C.c_double * 32), ("hvp_calls", C.c_int64),
                ("eval_calls", C.c_int64), ("seconds", C.c_double), ("kmeans_inertia", C.c_double)]


TUNE_MAX = 16


class TuneReport(C.Structure):
    _fields_ = [("n_candidates", C.c_int32), ("chosen", C.c_int32),
                ("edges_per_lane", C.c_int32 * TUNE_MAX), ("blocks_per_sm", C.c_int32 * TUNE_MAX),
                ("ms", C.c_double * TUNE_MAX)]


_vp = C.c_void_p
_SIGS = {
    "pspec_graph_create": (C.c_int, [C.c_int64, _vp, _vp, _vp, C.c_int, C.c_uint, _vp, C.POINTER(_vp)]),
    "pspec_graph_create_batched": (C.c_int, [C.c_int32, _vp, _vp, _vp, _vp, C.c_int, C.c_uint, _vp,
                                             C.POINTER(_vp)]),
    "pspec_graph_destroy": (None, [_vp]),
    "pspec_graph_info": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int32)]),
    "pspec_graph_status": (C.c_int, [_vp, _vp]),
    "pspec_eval": (C.c_int, [_vp, _vp, C.c_int, C.c_double, C.c_int, _vp, _vp, _vp, C.c_uint, _vp]),
    "pspec_hvp": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, C.c_int, _vp, C.c_uint, _vp]),
    "pspec_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
    "pspec_solve": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.POINTER(SolveOpts), C.c_int, _vp, _vp,
                              C.POINTER(C.c_double), C.POINTER(SolveStats), _vp]),
    "pspec_solve_batched": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.POINTER(SolveOpts), _vp, _vp, _vp,
                                      _vp, C.c_int, _vp]),
    "pspec_solve_lockstep": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.POINTER(SolveOpts), _vp, _vp, _vp,
                                       _vp, _vp, C.c_int, _vp]),
    "pspec_kmeans": (C.c_int, [_vp, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int,
                               C.c_int, _vp, _vp, C.POINTER(C.c_double), _vp]),
    "pspec_rcut": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(C.c_double), _vp]),
    "pspec_hvp_noalloc": (C.c_int, [C.c_int64, _vp, _vp, _vp, _vp, _vp, C.c_int, C.c_double, _vp,
                                    _vp]),
    "pspec_tune": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, C.c_int, C.POINTER(TuneReport), _vp]),
    "pspec_graph_create_shard": (C.c_int, [C.c_int64, C.c_int64, _vp, _vp, _vp, C.c_int, C.c_uint, _vp,
                                           C.POINTER(_vp)]),
    "pspec_eval_partial": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, _vp, _vp]),
    "pspec_eval_finish": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, _vp, _vp, _vp]),
    "pspec_hvp_partial": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, _vp, _vp, _vp]),
    "pspec_hvp_finish": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, _vp, _vp, C.c_uint, _vp]),
    "pspec_set_timing": (C.c_int, [_vp, C.c_int]),
    "pspec_kernel_times": (C.c_int, [_vp, C.c_char_p, C.c_size_t]),
    "pspec_last_error": (C.c_char_p, []),
    "pspec_version": (C.c_char_p, []),
}

_lib = None


class PspecError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libpspec.so once and declare every entry point."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2605_26975_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str, allow=(PSPEC_OK,)) -> int:
    if status not in allow:
        raise PspecError(status, where, lib().pspec_last_error().decode())
    return status


def declared_symbols():
    return sorted(_SIGS)
