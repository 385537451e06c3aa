"""Balanced-cut quality on Delaunay graphs of the unit square, the protocol of
the paper's Table 1 (Section 3.1): four clusters, RCut of spectral
clustering (the p = 2 stage: the span of the 4 smallest Laplacian
eigenvectors, then k-means) against RCut after the continuation in p, and
the relative reduction.

    python -m paper_2605_26975_gb300.table1 [--r 16 17 18 19] [--dtype f32|f64]

The graphs are drawn afresh (points uniform in the unit square, seeded), not
the collection's matrices, so the RCut values are comparable to the paper's
in size, not digit for digit.  Everything runs through the library's public
API on the current CUDA device.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(r: int, dtype: str = "f32", opts=None) -> dict:
    import torch

    from . import api
    from . import workloads as wl

    name = f"delaunay{r}"
    info = wl.WORKLOADS[name]
    g = wl.make_graph(name)
    k = info["k"]
    npdt = np.float32 if dtype == "f32" else np.float64
    U0 = torch.from_numpy(wl.orthonormal_block(2000 + info["index"], g.n, k, npdt)).cuda()
    G = api.Graph.from_csr(g)
    o = api.default_opts() if opts is None else opts
    t0 = time.perf_counter()
    _, _, rc_spec, st_spec, _ = G.solve(U0, [2.0], o)
    t_spec = time.perf_counter() - t0
    sched = list(info["p_schedule"])
    t0 = time.perf_counter()
    _, _, rc_p, st_p, status = G.solve(U0, sched, o)
    t_p = time.perf_counter() - t0
    return {"graph": name, "n": g.n, "nnz": g.nnz, "k": k, "dtype": dtype,
            "p_schedule": sched, "rcut_spec": rc_spec, "rcut_p": rc_p,
            "reduction_pct": 100.0 * (rc_p - rc_spec) / rc_spec,
            "seconds_spec": t_spec, "seconds_p": t_p,
            "newton_steps": sum(st_p["outer"]), "hvp_calls": st_p["hvp_calls"],
            "converged": status == 0}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--r", type=int, nargs="+", default=[16, 17, 18, 19])
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    for r in args.r:
        print(json.dumps(run(r, args.dtype)), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
