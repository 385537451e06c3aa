"""Exact Hessian vs Algorithm 1's sparse-plus-diagonal form inside the solve.

Algorithm 1 (Section 2) applies, per column, only the sparse-plus-diagonal
matrix (Hess N - lambda Hess D)/D; the exact Hessian of the quotient N/D adds
rank-two terms.  This runs the same solve (same U0, schedule, tolerances)
with each form and reports the truncated-CG iterations per stage, the
Newton steps, the final RCut and the time:

    python -m paper_2605_26975_gb300.ablation [--workload knn_gmm] [--dtype f32]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(workload: str, dtype: str = "f32") -> list:
    import torch

    from . import _abi, api
    from . import workloads as wl

    info = wl.WORKLOADS[workload]
    g = wl.make_graph(workload)
    k = info["k"]
    npdt = np.float32 if dtype == "f32" else np.float64
    U0 = torch.from_numpy(wl.orthonormal_block(2000 + info["index"], g.n, k, npdt)).cuda()
    G = api.Graph.from_csr(g)
    sched = list(info["p_schedule"])
    out = []
    for name, form in (("exact", _abi.PSPEC_HESSIAN_EXACT), ("alg1", _abi.PSPEC_HESSIAN_ALG1)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, rc, st, status = G.solve(U0, sched, api.default_opts(hessian_form=form))
        torch.cuda.synchronize()
        out.append({"workload": workload, "hessian": name, "dtype": dtype, "rcut": rc,
                    "tcg_iterations": st["inner"], "newton_steps": st["outer"],
                    "f": st["f"], "hvp_calls": st["hvp_calls"],
                    "seconds": time.perf_counter() - t0, "converged": status == 0})
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", nargs="+", default=["sbm4", "knn_gmm", "delaunay18"])
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    for w in args.workload:
        for line in run(w, args.dtype):
            print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
