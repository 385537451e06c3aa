"""ctypes binding of the all-core FP64 C oracle (plap_omp.c).

TEST INFRASTRUCTURE ONLY (see the package docstring): the tests pin it against
closed forms and the numpy oracle, and the benchmark's CPU-baseline leg times
it on every host core.  The library is compiled by ``build()`` (gcc, -O2,
OpenMP when the compiler has it; no fast-math, so every operation is IEEE
double) next to its source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "plap_omp.c")
LIB = os.path.join(HERE, "liboracle_omp.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle_omp.so (with OpenMP if gcc supports it)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp", "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: one thread
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed for plap_omp.c:\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        i64p, i32p, f64p = (np.ctypeslib.ndpointer(dtype=t, flags="C_CONTIGUOUS")
                            for t in (np.int64, np.int32, np.float64))
        L.oracle_threads.restype = C.c_int
        L.oracle_set_threads.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_eval.restype = C.c_int
        L.oracle_eval.argtypes = [C.c_int64, i64p, i32p, f64p, f64p, C.c_int, C.c_double,
                                  C.POINTER(C.c_double), f64p, f64p, C.c_void_p]
        L.oracle_hvp.restype = C.c_int
        L.oracle_hvp.argtypes = [C.c_int64, i64p, i32p, f64p, f64p, f64p, C.c_int, C.c_double,
                                 f64p, f64p]
        _lib = L
    return _lib


def threads() -> int:
    """OpenMP threads the oracle runs on (OMP_NUM_THREADS, else every core)."""
    return int(lib().oracle_threads())


def set_threads(t: int) -> int:
    """Run the following calls on t OpenMP threads; returns the count in effect."""
    return int(lib().oracle_set_threads(int(t)))


def _csr(g):
    return (np.ascontiguousarray(g.rowptr, dtype=np.int64), np.ascontiguousarray(g.col, dtype=np.int32),
            np.ascontiguousarray(g.val, dtype=np.float64))


def evaluate(g, U, p, grad=True, csr=None):
    """(F, N, D, gradient or None) of U (n x k, float64)."""
    rowptr, col, val = _csr(g) if csr is None else csr
    U = np.ascontiguousarray(U, dtype=np.float64)
    U2 = U[:, None] if U.ndim == 1 else U
    k = U2.shape[1]
    N, D = np.zeros(k), np.zeros(k)
    F = C.c_double()
    out = np.empty_like(U2) if grad else None
    st = lib().oracle_eval(g.n, rowptr, col, val, U2, k, float(p), C.byref(F), N, D,
                           out.ctypes.data if grad else None)
    if st != 0:
        raise ValueError("k must be in [1, 64]")
    return F.value, N, D, out


def hvp(g, U, V, p, csr=None, work=None):
    """Exact Euclidean Hessian of F_p at U applied to V (float64)."""
    rowptr, col, val = _csr(g) if csr is None else csr
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    U2 = U[:, None] if U.ndim == 1 else U
    V2 = V[:, None] if V.ndim == 1 else V
    k = U2.shape[1]
    out = np.empty_like(U2)
    delta = np.empty_like(U2) if work is None else work
    if lib().oracle_hvp(g.n, rowptr, col, val, U2, V2, k, float(p), out, delta) != 0:
        raise ValueError("k must be in [1, 64]")
    return out
