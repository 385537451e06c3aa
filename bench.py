"""Benchmark of the p-spectral clustering hot path on GB300.

One step = one pspec_eval (objective + gradient, keeping Delta_p u) and one
pspec_hvp (Hessian-vector product at the same U, reusing Delta_p u) on the
workload's graph -- the pattern of a Newton step, which evaluates once at U
and applies the Hessian at U: 2 * nnz * k edge-columns.  The metric is
edge-columns per second over the whole job (all ranks), with inputs resident
in HBM and the L2 flushed (a 256 MB write) before every timed step.
Alongside:
  roofline      the dominant kernel's algorithmic bytes per launch over its
                mean CUDA-event duration, against the measured HBM copy peak
  e2e           the same metric through the C ABI with host (pinned) buffers,
                host<->device copies inside the timed region
  cpu_baseline  the FP64 C oracle on every host core (OpenMP), full steps of
                the workload, plus a single-thread sample
  solve         wall time of the full solve down to the schedule's last p
                (FP32; with --solve both also the plain FP64 path), with RCut

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload grid3d]
                    [--impl ours|reference] [--solve none|f32|both]
Multi-GPU (torchrun): every rank runs an independent replica (its own seed);
there is no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2605_26975_gb300 import workloads as wl  # noqa: E402

P_BENCH = 1.3
METRIC = "p-Lap grad+HVP edge·col/s & % HBM peak; solve time to p=1.1 vs FP64 plain"
UNIT = "edge*col/s"
STEP = "pspec_eval (F + grad, Delta_p u kept) + pspec_hvp at the same U (Delta_p u reused)"
STEP_PLAIN = "pspec_eval (F + grad) + pspec_hvp"
L2_NOTE = "flushed (256 MB write) before every timed step"
L2_FLUSH_BYTES = 256 << 20
# the device code of the edge kernels: a profiles/ summary taken on other
# sources gives no traffic figure
KERNEL_SOURCES = ["paper_2605_26975_gb300/csrc/edge_kernels.cuh",
                  "paper_2605_26975_gb300/csrc/edge_staged.cuh",
                  "paper_2605_26975_gb300/csrc/common.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: enough for about 2 s of timed region, at least 50)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="grid3d",
                    choices=["knn_gmm", "grid3d", "dcsbm", "sbm4", "sbm_batch"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--solve", default="f32", choices=["none", "f32", "both"],
                    help="full solve to the schedule's last p: FP32 only, or FP32 and plain FP64")
    ap.add_argument("--solve-gtol", type=float, default=None,
                    help="relative gradient tolerance of every stage (library default 1e-6)")
    ap.add_argument("--solve-max-outer", type=int, default=None,
                    help="Newton steps allowed per stage (library default 30)")
    ap.add_argument("--no-solve", action="store_true", help="same as --solve none")
    ap.add_argument("--solve-perturbed", action="store_true",
                    help="with --solve both: also the FP64 solve from U0 perturbed at FP32 rounding")
    ap.add_argument("--no-keep", action="store_true",
                    help="plain pspec_hvp (the HVP kernel writes Delta_p u again)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--eager", action="store_true", help="launch the step's kernels one by one")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (no pspec_tune)")
    return ap.parse_args()


def describe(name, n, nnz, k):
    desc = {
        "knn_gmm": "kNN similarity graph: 200,000 points, 8 isotropic 2-D Gaussians, 10-NN symmetrised, w=exp(-d^2/0.25)",
        "grid3d": "3-D 200^3 6-neighbour grid, w~U[0.5,1.5], 0.1% long-range links",
        "dcsbm": "degree-corrected SBM, n=1,000,000, 16 blocks, Pareto(2.5) degrees, w~U[0.1,1]",
        "sbm4": "SBM n=1,000, 4 blocks, p_in 0.05, p_out 0.002",
        "sbm_batch": "512 SBMs, n log-uniform in [500, 50,000], 2..8 blocks, mean degree 8..20, "
                     "k in {2,4,8}; one batched handle per k",
    }[name]
    return f"{desc} (n={n}, nnz={nnz}, k={k})"


class Part:
    """One graph handle of the workload: its CSR (a batch's concatenation for
    sbm_batch), vertex offsets of the graphs in it, and the blocks U, V."""

    def __init__(self, csr, node_off, graphs, U, V, k):
        self.csr, self.node_off, self.graphs, self.U, self.V, self.k = csr, node_off, graphs, U, V, k

    def edge_cols(self):
        return 2 * self.csr.nnz * self.k

    def samples(self):
        """(graph, U rows, V rows) of every graph in the part."""
        if self.node_off is None:
            return [(self.csr, self.U, self.V)]
        o = self.node_off
        return [(g, self.U[o[i]:o[i + 1]], self.V[o[i]:o[i + 1]]) for i, g in enumerate(self.graphs)]


def build_parts(name, rank=0):
    """The workload as a list of Parts; sbm_batch is grouped by k (a handle
    holds graphs of one k), every other workload is one graph."""
    info = wl.WORKLOADS[name]
    if name == "sbm_batch":
        gs, us, vs = replica_seeds(name, rank)
        batch = wl.make_graph(name) if rank == 0 else wl.sbm_batch(gs)
        parts = []
        for k in (2, 4, 8):
            idx = np.flatnonzero(batch.k == k)
            sub = wl.concat_graphs([batch.graphs[i] for i in idx], [k] * idx.size)
            n = sub.csr.n
            parts.append(Part(sub.csr, sub.node_off, sub.graphs, wl.orthonormal_block(us + 10 * k, n, k),
                              wl.gaussian_block(vs + 10 * k, n, k), k))
        return parts, info
    g, U, V, info = build_workload(name, seed_shift=rank)
    return [Part(g, None, None, U, V, info["k"])], info


def q_of(k):
    """Column lanes per row of the edge kernels for k columns (as the library)."""
    return 4 if (k % 4 == 0 and k // 4 >= 4) else 2 if (k % 2 == 0 and k // 2 >= 4) else 1


def staged_max_entries(k):
    """Most entries per warp task the staged edge kernel takes for k columns."""
    return min(256, 8192 // (8 * k))


def bytes_eval_edges(g, k):
    """Algorithmic bytes of the objective's edge kernel: the matrix (column
    index + weight per entry), the row offsets, U in and Delta_p u out."""
    return g.nnz * 8 + (g.n + 1) * 8 + 2 * g.n * k * 4


def bytes_hvp_edges(g, k):
    """Algorithmic bytes of the Hessian product's edge kernel: the matrix, the
    row offsets, U and V in, the sparse part out (Delta_p u is the
    objective's, kept from the evaluation at the same U)."""
    return g.nnz * 8 + (g.n + 1) * 8 + 3 * g.n * k * 4


def source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(kernel, workload):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            key, _, v = line.partition("=")
            vals[key.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_ready(self, timeout=10.0):
        """Block until the first sample arrives (nvidia-smi takes a moment to start)."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()

    def summary(self, t0, t1):
        """Median SM clock, max clock and active throttle reasons of the samples
        that arrived between host times t0 and t1."""
        if self.proc is None:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if not t0 <= ts <= t1:
                continue
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": []}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_throughput(ms_local, edge_cols_local, dist=None):
    """Whole-job throughput of independent replicas: every rank's step time is
    reduced with MAX (the job is as slow as its slowest rank) and the units
    of all ranks are summed.  Returns (value, ms_max)."""
    import torch
    world = 1
    ms = float(ms_local)
    units = float(edge_cols_local)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([units], dtype=torch.float64, device=dev)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = t.item(), u.item()
    return units / (ms * 1e-3), ms


def replica_seeds(name, rank):
    """Graph and block seeds of rank `rank`'s replica (rank 0: the named workload)."""
    idx = wl.WORKLOADS[name]["index"]
    return 1000 + idx + 100 * rank, 2000 + idx + 100 * rank, 3000 + idx + 100 * rank


def workload_desc(name, parts):
    n = sum(pt.csr.n for pt in parts)
    nnz = sum(pt.csr.nnz for pt in parts)
    ks = "/".join(str(pt.k) for pt in parts)
    return describe(name, n, nnz, ks)


def build_workload(name, seed_shift=0):
    info = wl.WORKLOADS[name]
    if seed_shift == 0:
        g = wl.make_graph(name)
        U, V = wl.make_blocks(name, g.n, info["k"])
    else:  # an independent replica for rank > 0
        gs, us, vs = replica_seeds(name, seed_shift)
        g = {"knn_gmm": lambda s: wl.knn_gaussian_mixture(s),
             "grid3d": lambda s: wl.grid3d_longrange(s),
             "dcsbm": lambda s: wl.dcsbm_powerlaw(s),
             "sbm4": lambda s: wl.sbm_bernoulli(s)}[name](gs)
        U = wl.orthonormal_block(us, g.n, info["k"])
        V = wl.gaussian_block(vs, g.n, info["k"])
    return g, U, V, info


def oracle_items(parts):
    """(graph, CSR as the C oracle takes it, U, V in FP64, k) of every graph of
    the workload."""
    items = []
    for part in parts:
        for g, U, V in part.samples():
            csr = (np.ascontiguousarray(g.rowptr, dtype=np.int64),
                   np.ascontiguousarray(g.col, dtype=np.int32),
                   np.ascontiguousarray(g.val, dtype=np.float64))
            items.append((g, csr, U.astype(np.float64), V.astype(np.float64), part.k))
    return items


def oracle_steps(items, p, budget_s, max_steps):
    """The FP64 C oracle as it stands: objective + gradient and the Hessian
    product on the workload's graphs in order (cycling) until budget_s
    seconds or max_steps graph-steps pass.  Returns (edge-columns done,
    seconds, graph-steps)."""
    from oracle import omp
    t0 = time.perf_counter()
    done = steps = 0
    while True:
        g, csr, U64, V64, k = items[steps % len(items)]
        omp.evaluate(g, U64, p, csr=csr)
        omp.hvp(g, U64, V64, p, csr=csr)
        done += 2 * g.nnz * k
        steps += 1
        if time.perf_counter() - t0 > budget_s or steps >= max_steps:
            break
    return done, time.perf_counter() - t0, steps


class RowBlock:
    """The first `rows` rows of a graph (all columns kept): a bounded sample of
    its work for the single-thread oracle."""

    def __init__(self, g, rows):
        self.n = rows
        self.nnz = int(g.rowptr[rows])


def single_thread_sample(items, p, edge_cols=4_000_000):
    """The C oracle on one thread, one objective + gradient + Hessian product
    over a row block of the first graph with about edge_cols edge-columns."""
    from oracle import omp
    g, csr, U64, V64, k = items[0]
    rows = int(np.searchsorted(csr[0], edge_cols // (2 * k), side="right")) - 1
    rows = max(1, min(g.n, rows))
    blk = RowBlock(g, rows)
    sub = (csr[0][:rows + 1], csr[1][:blk.nnz], csr[2][:blk.nnz])
    omp.set_threads(1)
    try:
        t0 = time.perf_counter()
        omp.evaluate(blk, U64, p, csr=sub)
        omp.hvp(blk, U64, V64, p, csr=sub)
        dt = time.perf_counter() - t0
    finally:
        omp.set_threads(os.cpu_count() or 1)
    return {"value": 2 * blk.nnz * k / dt, "cores": 1,
            "sample": f"one eval+grad+HVP of rows 0..{rows} ({blk.nnz} entries, k={k}) "
                      f"of the first graph, {dt:.2f} s"}


def cpu_baseline(parts, p, budget_s=15.0):
    """The FP64 C oracle on every host core (OpenMP over rows), full steps of
    the workload for about budget_s seconds, plus a single-thread sample."""
    from oracle import omp
    items = oracle_items(parts)
    cores = omp.set_threads(os.cpu_count() or 1)
    oracle_steps(items[:1], p, 0.0, 1) if items[0][0].nnz < 50_000_000 else None  # warm-up
    max_steps = 20 if len(items) == 1 else 100_000
    done, dt, steps = oracle_steps(items, p, budget_s, max_steps)
    what = "full eval+grad+HVP step(s)" if len(items) == 1 else "graphs' eval+grad+HVP steps"
    return {"value": done / dt, "unit": "edge*col/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} {what} of the FP64 C oracle (OpenMP, {cores} threads) on this "
                      f"workload, {dt:.1f} s",
            "single_thread": single_thread_sample(items, p)}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from oracle import omp
    parts, info = build_parts(args.workload)
    items = oracle_items(parts)
    cores = omp.set_threads(os.cpu_count() or 1)
    # each timed step is one oracle eval+grad+HVP of the workload's graph (of
    # up to 40 of a batch's graphs); keep the run to a few minutes
    steps = max(1, min(args.steps or 5, 8))
    per_step = 1 if len(items) == 1 else 40
    oracle_steps(items, P_BENCH, 0.0, 1)  # warm-up
    done, dt, _ = oracle_steps(items, P_BENCH, float("inf"), steps * per_step)
    value = done / dt
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": 1, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(args.workload, parts),
                                            "p": P_BENCH,
                                            "step": "objective + gradient, then the Hessian "
                                                    "product at the same U (FP64 C oracle)",
                                            "l2": "n/a (FP64 oracle on the host cores)",
                                            "parallelism": f"replicas x{args.gpus}"},
            "cpu_baseline": {"value": value, "unit": "edge*col/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} step(s) of {per_step} graph eval+grad+HVP of the "
                                       f"FP64 C oracle (OpenMP, {cores} threads)"},
            "e2e": {"value": value, "unit": "edge*col/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    import torch
    import torch.distributed as dist

    from paper_2605_26975_gb300 import api, build
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    parts, info = build_parts(args.workload, rank)
    for pt in parts:
        pt.G = api.Graph(pt.csr.rowptr, pt.csr.col, pt.csr.val, node_off=pt.node_off)
        pt.Ud = torch.from_numpy(pt.U).cuda()
        pt.Vd = torch.from_numpy(pt.V).cuda()
        pt.grad = torch.empty_like(pt.Ud)
        pt.HV = torch.empty_like(pt.Ud)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # a batched handle keeps no Delta_p u: its step is the plain pair
    keep = not args.no_keep and all(pt.G.n_graphs == 1 for pt in parts)

    def step():
        for pt in parts:
            pt.G.eval(pt.Ud, P_BENCH, grad_out=pt.grad, keep_delta=keep)
            pt.G.hvp(pt.Ud, pt.Vd, P_BENCH, out=pt.HV, delta_kept=keep)

    # launch shape per handle from the autotuner (edges per lane, blocks per SM)
    tuned = []
    for pt in parts:
        if not args.no_tune:
            cands, best = pt.G.tune(pt.Ud, pt.Vd, P_BENCH, reps=3)
            L, b, ms = cands[best]
            tuned.append({"k": pt.k, "edges_per_lane": L, "blocks_per_sm": b,
                          "kernel": "staged" if 32 * L // q_of(pt.k) <= staged_max_entries(pt.k) else "direct",
                          "eval_hvp_ms": round(ms, 4),
                          "candidates": [[c[0], c[1], round(c[2], 4)] for c in cands]})
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    for pt in parts:
        assert pt.G.status() == 0
    # the step (per handle eval + hvp: 4 kernel launches, 6 for a batch)
    # replayed as one CUDA graph, so host launch latency does not sit between
    # the kernels
    graph = None
    if not args.eager:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()
        run_step = graph.replay
    else:
        run_step = step

    if args.steps is None:  # about 2 s of timed region, from five timed steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            flush.zero_()
            run_step()
        e1.record(stream)
        torch.cuda.synchronize()
        per_step = e0.elapsed_time(e1) / 5
        args.steps = int(min(20000, max(50, 2000.0 / max(per_step, 1e-3))))
        if world > 1:  # every rank times the same number of steps: rank 0's
            kt = torch.tensor([args.steps], dtype=torch.int64, device="cuda")
            dist.broadcast(kt, 0)
            args.steps = int(kt.item())

    # ---- timed region: device time of every step, L2 flushed before each
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    sampler.wait_ready()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        run_step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    wall = wall1 - wall0
    if world > 1:
        dist.barrier()
    clocks = sampler.summary(wall0, wall1)
    if clocks is not None and clocks["samples"] == 0:
        # a region shorter than the sampling period: keep the GPU under the same
        # step loop for one more second and report the samples of both
        while time.perf_counter() - wall1 < 1.0:
            for _ in range(20):
                flush.zero_()
                run_step()
            torch.cuda.synchronize()
        clocks = sampler.summary(wall0, time.perf_counter())
        if clocks is not None:
            clocks["window"] = "timed region + 1 s of the same step loop right after it"
    sampler.stop()
    ms_local = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    edge_cols = sum(pt.edge_cols() for pt in parts)
    value, ms = job_throughput(ms_local, edge_cols, dist if world > 1 else None)

    # ---- per-kernel device times (same steps, library events on the stream)
    for pt in parts:
        pt.G.set_timing(True)
    for _ in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    times = {}
    for pt in parts:
        for name, (c, t) in pt.G.kernel_times().items():
            c0, t0 = times.get(name, (0, 0.0))
            times[name] = (c0 + c, t0 + t)
        pt.G.set_timing(False)
    launches = sum(c for c, _ in times.values()) // args.steps
    shares = {name: t for name, (c, t) in times.items()}
    dom = max(shares, key=shares.get)
    dom_launches, dom_ms = times[dom]
    byte_fn = {"hvp_edges": bytes_hvp_edges, "eval_edges": bytes_eval_edges}.get(dom)
    peak, peak_kind = measured_peak()
    roofline = None
    if byte_fn is not None:
        algo_step = sum(byte_fn(pt.csr, pt.k) for pt in parts)  # one launch per handle
        achieved = algo_step * args.steps / (dom_ms * 1e-3) / 1e9
        roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                    "traffic": read_traffic(dom, args.workload) if len(parts) == 1 else None,
                    "algorithmic_bytes_per_launch": algo_step / len(parts),
                    "launches_per_step": len(parts),
                    "mean_launch_ms": dom_ms / dom_launches,
                    "kernel_ms_per_step": {n: t / args.steps for n, (c, t) in times.items()}}

    # ---- e2e through the C ABI with pinned host buffers
    for pt in parts:
        pt.Uh = torch.from_numpy(pt.U).pin_memory()
        pt.Vh = torch.from_numpy(pt.V).pin_memory()
        pt.gh = torch.empty_like(pt.Uh).pin_memory()
        pt.hh = torch.empty_like(pt.Uh).pin_memory()

    def host_step():
        for pt in parts:
            pt.G.eval_host(pt.Uh, P_BENCH, pt.gh, keep_delta=keep)
            pt.G.hvp_host(pt.Uh, pt.Vh, P_BENCH, pt.hh, delta_kept=keep)

    for _ in range(2):
        host_step()
    e2e_steps = max(3, min(args.steps // 2, 100))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        flush.zero_()
        host_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    blk = sum(pt.csr.n * pt.k * 4 for pt in parts)
    n_f = sum(pt.G.n_graphs for pt in parts)
    e2e = {"value": world * edge_cols / e2e_s, "unit": "edge*col/s",
           "h2d_bytes_per_step": 3 * blk, "d2h_bytes_per_step": 2 * blk + 8 * n_f,
           "note": "wall clock per step incl. a 256 MB L2 flush; copies and kernels synchronous"}

    # ---- full solve to the last p (FP32; with --solve both the plain FP64 path too)
    solve = None
    if args.no_solve:
        args.solve = "none"
    if args.solve != "none" and rank == 0 and len(parts) == 1:
        pt = parts[0]
        sched = list(info["p_schedule"])
        kw = {}
        if args.solve_gtol is not None:
            kw["gtol_rel"] = args.solve_gtol
        if args.solve_max_outer is not None:
            kw["max_outer"] = args.solve_max_outer
        opts = api.default_opts(**kw)
        cap = opts.max_outer

        def run_solve(U0):
            t0 = time.perf_counter()
            _, lab, rc, st, status = pt.G.solve(U0, sched, opts)
            dt = time.perf_counter() - t0
            return {"s": dt, "rcut": rc, "hvp_calls": st["hvp_calls"],
                    "newton_steps": sum(st["outer"]), "stages_at_cap": sum(o >= cap for o in st["outer"]),
                    "f": st["f"], "status": status}

        solve = {"p_schedule": sched, "gtol_rel": opts.gtol_rel, "max_outer": cap,
                 "f32": run_solve(pt.Ud)}
        if args.solve == "both":
            solve["f64"] = run_solve(torch.from_numpy(pt.U.astype(np.float64)).cuda())
            solve["speedup"] = solve["f64"]["s"] / solve["f32"]["s"]
            solve["rcut_rel_diff"] = abs(solve["f32"]["rcut"] - solve["f64"]["rcut"]) / solve["f64"]["rcut"]
        if args.solve == "both" and args.solve_perturbed:
            # the same FP64 solve from U0 perturbed at FP32's rounding level
            # (each entry times 1 + 2^-24 s, s = +-1 seeded): how far apart two
            # FP64 paths end from starting points as close as FP32 rounding
            sgn = np.where(np.random.default_rng(7).random(pt.U.shape) < 0.5, -1.0, 1.0)
            U0p = pt.U.astype(np.float64) * (1.0 + 2.0 ** -24 * sgn)
            solve["f64_perturbed"] = run_solve(torch.from_numpy(U0p).cuda())
            solve["rcut_rel_diff_f64_perturbed"] = (abs(solve["f64_perturbed"]["rcut"] - solve["f64"]["rcut"])
                                                    / solve["f64"]["rcut"])

    if args.solve != "none" and rank == 0 and len(parts) > 1:
        # the batch: every graph its own solve, all graphs of a k-handle in
        # lockstep (pspec_solve_lockstep, FP32); with --solve both also the
        # per-graph concurrent solves (pspec_solve_batched) for comparison
        sched = list(info["p_schedule"])

        # each graph's U0: orthonormal columns on its own rows, as the solve expects
        U0s = [torch.from_numpy(np.concatenate([wl.orthonormal_block(2000 + 10 * pt.k + i, g.n, pt.k)
                                                for i, g in enumerate(pt.graphs)])).cuda() for pt in parts]

        def run_batch(kind):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if kind == "lockstep":
                # the k-handles concurrently, each on its own solve stream
                from concurrent.futures import ThreadPoolExecutor
                with ThreadPoolExecutor(len(parts)) as ex:
                    outs = list(ex.map(lambda a: a[0].G.solve_lockstep(a[1], sched, api.default_opts(),
                                                                       allow_errors=True),
                                       zip(parts, U0s)))
                rcuts = [o[2] for o in outs]
                stat = [o[3] for o in outs]
                newton = [sum(sum(x["outer"]) for x in o[4]) for o in outs]
                tcg = [sum(x["hvp_calls"] for x in o[4]) for o in outs]
            else:
                rcuts, stat, newton, tcg = [], [], [], []
                for pt, U0 in zip(parts, U0s):
                    _, _, rc, status, _ = pt.G.solve_batched(U0, sched, api.default_opts())
                    rcuts.append(rc)
                    stat.append(status)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0, np.concatenate(rcuts), np.concatenate(stat),
                    int(sum(newton)), int(sum(tcg)))

        t_ls, rc_ls, st_ls, newton, tcg = run_batch("lockstep")
        solve = {"p_schedule": sched, "lockstep_f32_s": t_ls, "graphs": int(rc_ls.size),
                 "graphs_ok_or_capped": int(np.isin(st_ls, (0, 6)).sum()),
                 "rcut_median": float(np.nanmedian(rc_ls)), "rcut_max": float(np.nanmax(rc_ls)),
                 "newton_steps": newton, "tcg_iterations": tcg,
                 "note": "one pspec_solve_lockstep call per k-handle, the three handles on host "
                         "threads: every graph's Newton/tCG decisions on the device, one launch per "
                         "step for the whole handle; k-means per graph on 16 host threads"}
        if args.solve == "both":
            t_b, rc_b, st_b, _, _ = run_batch("batched")
            rel = np.abs(rc_ls - rc_b) / rc_b
            solve.update({"batched_f32_s": t_b, "speedup_lockstep_vs_batched": t_b / t_ls,
                          "rcut_rel_diff_median": float(np.nanmedian(rel)),
                          "graphs_rcut_within_1pct": int(np.sum(rel <= 0.01))})

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(parts, P_BENCH)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, parts), "p": P_BENCH,
                       "step": (STEP if keep else STEP_PLAIN) + (" per handle" if len(parts) > 1 else "")
                               + ("" if args.eager else ", replayed as a CUDA graph"),
                       "l2": L2_NOTE,
                       "launch_shape": tuned if tuned else "default (not tuned)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches * args.steps, "solve": solve,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
