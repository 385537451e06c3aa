"""The C-ABI library builds, loads and exports every entry point that
include/pspec.h declares; argument validation that happens before any device
work returns the documented status without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pspec.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2605_26975_gb300 import build, _abi
    build.build()
    return _abi.lib()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pspec_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["pspec_graph_create", "pspec_graph_create_batched", "pspec_graph_destroy",
                     "pspec_eval", "pspec_hvp", "pspec_solve", "pspec_kmeans", "pspec_rcut",
                     "pspec_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2605_26975_gb300 import _abi
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(_abi.declared_symbols())


def test_version_and_defaults(lib):
    from paper_2605_26975_gb300 import _abi
    assert b"sm_103a" in lib.pspec_version()
    o = _abi.SolveOpts()
    lib.pspec_solve_opts_default(C.byref(o))
    assert o.max_outer == 30 and o.max_inner == 50 and o.kappa == 0.1 and o.theta == 1.0
    assert o.kmeans_restarts == 10 and o.kmeans_max_iter == 300


def _create(lib, n, rowptr, col, val, flags=1):
    from paper_2605_26975_gb300 import _abi
    h = C.c_void_p()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    st = lib.pspec_graph_create(n, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                                _abi.PSPEC_F32, flags, None, C.byref(h))
    return st, h


@pytest.mark.parametrize("case", ["n0", "rowptr0", "decreasing", "col_range", "negative", "nan",
                                  "asym"])
def test_graph_create_rejects_bad_csr_on_host(lib, case):
    from paper_2605_26975_gb300 import _abi
    n, rowptr, col, val = 3, [0, 1, 3, 4], [1, 0, 2, 1], [1.0, 1.0, 2.0, 2.0]
    flags = _abi.PSPEC_HOST_PTRS
    if case == "n0":
        n = 0
    elif case == "rowptr0":
        rowptr = [1, 1, 3, 4]
    elif case == "decreasing":
        rowptr = [0, 2, 1, 4]
    elif case == "col_range":
        col = [1, 0, 3, 1]
    elif case == "negative":
        val = [1.0, 1.0, -2.0, 2.0]
    elif case == "nan":
        val = [1.0, float("nan"), 2.0, 2.0]
    elif case == "asym":
        val = [1.0, 1.0, 2.0, 3.0]
        flags |= _abi.PSPEC_CHECK_SYMMETRY
    st, h = _create(lib, n, rowptr, col, val, flags)
    assert st == _abi.PSPEC_ERR_INVALID_ARG
    assert not h.value
    assert lib.pspec_last_error()


def test_calls_reject_null_graph_and_bad_arguments(lib):
    from paper_2605_26975_gb300 import _abi
    F = C.c_double()
    assert lib.pspec_eval(None, None, 4, 1.5, 0, C.byref(F), None, None, 0, None) == _abi.PSPEC_ERR_INVALID_ARG
    assert lib.pspec_hvp(None, None, None, 4, 1.5, 0, None, 0, None) == _abi.PSPEC_ERR_INVALID_ARG
    sched = np.array([2.0, 1.5])
    assert lib.pspec_solve(None, 4, sched.ctypes.data, 2, None, 0, None, None, None, None,
                           None) == _abi.PSPEC_ERR_INVALID_ARG
    inertia = C.c_double()
    assert lib.pspec_kmeans(None, 10, 2, 0, 2, 0, 1, 10, None, None, C.byref(inertia),
                            None) == _abi.PSPEC_ERR_INVALID_ARG
    out = C.c_double()
    assert lib.pspec_rcut(None, None, 2, C.byref(out), None) == _abi.PSPEC_ERR_INVALID_ARG
    lib.pspec_graph_destroy(None)  # accepted


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the option, statistics and tuning structs have the
    C layout of include/pspec.h: sizes and every field offset, printed by a C
    program compiled against the header."""
    import shutil
    import subprocess
    from paper_2605_26975_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pspec_solve_opts": _abi.SolveOpts, "pspec_solve_stats": _abi.SolveStats,
               "pspec_tune_report": _abi.TuneReport}
    lines = ['#include <stdio.h>', '#include "pspec.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
