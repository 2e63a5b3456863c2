#!/usr/bin/env python3
"""GSL-LPA benchmark: LPA + split throughput (|E|/s) on one GB300 per rank.

Default workload: R-MAT scale 25, edge factor 24 (a, b, c, d = 0.57, 0.19,
0.19, 0.05), symmetrised, deduplicated, self-loops dropped, vertex ids
randomly permuted, unit weights; synchronous LPA, tolerance 0.05, at most 20
sweeps, then the split.  |E| counts directed CSR entries (both directions of
every edge).  One step = one gsl_gsllpa call (all sweeps + split) on the
resident graph.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own copy of the graph on its own
GPU (the single-graph path does not shard; replicas only, no collective on
the data path); value = all ranks' entries / max-over-ranks step time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LPA+split |E|/s on R-MAT-25 (sync, tol 0.05, max 20 sweeps)"
UNIT = "edges/s"


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--scale", type=int, default=25, help="R-MAT scale of the workload")
    p.add_argument("--edge-factor", type=int, default=24)
    p.add_argument("--mode", choices=["sync", "async"], default="sync")
    p.add_argument("--weights", choices=["unit", "int", "f32"], default="unit",
                   help="edge weights: unit (the benchmark), int32 1..32 or float32 k/8 for k in 1..32, "
                        "both from a hash of the endpoint pair (symmetric)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cache", default=default_cache())
    p.add_argument("--profile-json", default="", help="also write the per-slot profile here")
    p.add_argument("--workload", choices=["rmat", "batched", "served", "compare"], default="rmat",
                   help="rmat: one R-MAT graph (default); batched: many SBM graphs per call vs one call per graph")
    p.add_argument("--graphs", type=int, default=4096, help="graphs in the batched workload")
    p.add_argument("--gen-procs", type=int, default=0, help="host processes generating the batched graphs")
    p.add_argument("--rate", type=float, default=2000.0, help="served: mean Poisson arrival rate (requests/s)")
    p.add_argument("--duration", type=float, default=60.0, help="served: seconds of arrivals per rate")
    p.add_argument("--pool", type=int, default=512, help="served: distinct request graphs (drawn with replacement)")
    p.add_argument("--line-served-duration", type=float, default=10.0,
                   help="seconds of arrivals per rate of the served object in the default line")
    p.add_argument("--no-batched", action="store_true", help="default line without the batched object")
    p.add_argument("--no-served", action="store_true", help="default line without the served object")
    p.add_argument("--slots", type=int, default=3, help="served: concurrent batches of the server")
    return p.parse_args()


# ------------------------------------------------------------------- ranks
def rank_env():
    """(rank, world, local_rank) from the launcher's environment (torchrun
    sets RANK / WORLD_SIZE / LOCAL_RANK; a plain run is rank 0 of 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device="cpu"):
    """The largest of every rank's x (each rank passes its own step time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(world, units_per_rank, ms):
    """Whole-job throughput of `world` replicas that each process
    units_per_rank units, timed by the slowest rank (ms)."""
    return world * units_per_rank / (ms * 1e-3)


# ------------------------------------------------------------------ workload
def workload_paths(scale, edge_factor, cache):
    """The .npy files (offsets, cols) of the cached R-MAT workload graph."""
    tag = f"rmat{scale}_ef{edge_factor}_s1"
    return os.path.join(cache, tag + "_offsets.npy"), os.path.join(cache, tag + "_cols.npy")


def default_cache():
    return os.environ.get("GSL_BENCH_CACHE", os.path.join(tempfile.gettempdir(), "gsl_bench_cache"))


def workload_graph(scale, edge_factor, cache, rank, world):
    """R-MAT graph, generated once per machine and cached as .npy files."""
    import numpy as np
    import inputs as I
    off_p, col_p = workload_paths(scale, edge_factor, cache)
    if rank == 0 and not (os.path.exists(off_p) and os.path.exists(col_p)):
        os.makedirs(cache, exist_ok=True)
        t0 = time.time()
        g = I.rmat(scale, edge_factor, 0.57, 0.19, 0.19, seed=1, permute=True)
        gen_s = time.time() - t0
        for p_, a in ((off_p, g.offsets), (col_p, g.cols)):
            tmp = p_ + f".{os.getpid()}.tmp.npy"
            np.save(tmp, a)
            os.replace(tmp, p_)
        print(f"[bench] generated {g} in {gen_s:.1f}s", file=sys.stderr, flush=True)
        del g
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    offsets = np.load(off_p, mmap_mode="r")
    cols = np.load(col_p, mmap_mode="r")
    return offsets, cols


def edge_weights(off, col, kind):
    """Symmetric synthetic weights on the device: a hash of the unordered
    endpoint pair picks k in 1..32; int32 k or float32 k/8 (exact in float64
    sums)."""
    import torch
    n = off.numel() - 1
    rows = torch.repeat_interleave(torch.arange(n, device=off.device, dtype=torch.int64), off[1:] - off[:-1])
    a = torch.minimum(rows, col.to(torch.int64))
    b = torch.maximum(rows, col.to(torch.int64))
    del rows
    h = (a * 0x9E3779B1 + b * 0x85EBCA6B) & 0xFFFFFFFF
    h = (h ^ (h >> 15)) * 0x2C1B3C6D & 0xFFFFFFFF
    k = ((h >> 11) & 31) + 1
    del a, b, h
    return k.to(torch.int32) if kind == "int" else (k.to(torch.float32) / 8.0)


# -------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- CPU side
def oracle_gsllpa(offsets, cols, tol, max_iters):
    """The oracle as it stands (single thread): synchronous lpa() of
    Algorithm 3, then the BFS split of Algorithm 2, timed per phase."""
    import inputs as I
    import oracle as O
    g = I.Graph(offsets, cols)
    t0 = time.perf_counter()
    lab, t, dn = O.lpa_sync(g, tol, max_iters)
    t1 = time.perf_counter()
    split = O.split_bfs(g, lab)
    t2 = time.perf_counter()
    return split, t, dn, t1 - t0, t2 - t1


def cpu_baseline(offsets, cols, tol, max_iters, workload, gpu_labels=None, gpu_changed=None):
    """The oracle on the benchmark's own graph (the whole workload, one
    thread), beside the GPU result: also reports whether the GPU's labels
    and per-sweep change counts equal the oracle's."""
    split, t, dn, lpa_s, split_s = oracle_gsllpa(offsets, cols, tol, max_iters)
    n, nnz = offsets.shape[0] - 1, cols.shape[0]
    out = {
        "value": nnz / (lpa_s + split_s), "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": (f"the whole workload ({workload}, n={n}, nnz={nnz}): oracle GSL-LPA (Jacobi LPA tol {tol} "
                   f"max {max_iters}, then BFS split), {t} sweeps, lpa {lpa_s:.1f}s split {split_s:.1f}s, "
                   f"one thread"),
        "host_cores": os.cpu_count(),
        "seconds": lpa_s + split_s,
    }
    if gpu_labels is not None:
        import numpy as np
        out["labels_identical_to_gpu"] = bool(np.array_equal(split, gpu_labels))
        out["changed_identical_to_gpu"] = list(map(int, dn)) == list(gpu_changed or [])
    return out


REF_SCALE = 21     # R-MAT scale of one reference-arm step


def run_reference(args):
    """The oracle timed as the reference arm: each step is one full oracle
    GSL-LPA (Jacobi LPA + BFS split, one thread) on an R-MAT graph of the
    workload's generator and parameters at scale REF_SCALE (1/16 of the
    scale-25 workload: 25 steps of the full graph would take most of an
    hour)."""
    rank = rank_env()[0]
    if rank != 0:
        return 0
    import inputs as I
    import oracle  # noqa: F401  (builds the oracle)
    scale = min(args.scale, REF_SCALE)
    g = I.rmat(scale, args.edge_factor, 0.57, 0.19, 0.19, seed=1, permute=True)
    vals, info = [], None
    for i in range(args.warmup + args.steps):
        _, t, _, lpa_s, split_s = oracle_gsllpa(g.offsets, g.cols, 0.05, 20)
        if i >= args.warmup:
            vals.append(g.nnz / (lpa_s + split_s))
        info = (t, lpa_s, split_s)
    value = statistics.median(vals) if vals else 0.0
    sample = (f"per step the oracle's full GSL-LPA (Jacobi LPA tol 0.05 max 20, then BFS split, one thread) on "
              f"R-MAT scale {scale} ef {args.edge_factor} of the same generator and seed: n={g.n}, nnz={g.nnz}, "
              f"{info[0] if info else 0} sweeps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale}-ef{args.edge_factor}", "sample_scale": scale,
                   "tolerance": 0.05, "max_iters": 20, "mode": "sync"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- batched mode
def _gen_batched(args_):
    g0, g1 = args_
    import inputs as I
    out = []
    for g in range(g0, g1):
        gr = I.batched_sbm(g, threads=1)
        out.append((gr.offsets, gr.cols))
    return out


def batched_graphs(count, procs):
    """The batched workload: graph g is the planted partition with the batched
    parameter laws and seed g (inputs.batched_sbm_params)."""
    import multiprocessing as mp
    procs = procs or max(1, min(32, os.cpu_count() or 1))
    chunks = [(k * count // procs, (k + 1) * count // procs) for k in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_gen_batched, chunks)
    return [g for part in parts for g in part]


def pack_graphs(graphs):
    """Disjoint union of (offsets, cols) pairs as one CSR: (offsets, cols, vptr)."""
    import numpy as np
    G = len(graphs)
    vptr = np.zeros(G + 1, dtype=np.int64)
    eptr = np.zeros(G + 1, dtype=np.int64)
    for k, (o, c) in enumerate(graphs):
        vptr[k + 1] = vptr[k] + (o.shape[0] - 1)
        eptr[k + 1] = eptr[k] + c.shape[0]
    off_u = np.empty(int(vptr[-1]) + 1, dtype=np.int64)
    col_u = np.empty(int(eptr[-1]), dtype=np.int32)
    off_u[0] = 0
    for k, (o, c) in enumerate(graphs):
        off_u[vptr[k] + 1:vptr[k + 1] + 1] = o[1:] + eptr[k]
        col_u[eptr[k]:eptr[k + 1]] = c + vptr[k]
    return off_u, col_u, vptr


TUNE_SAMPLE = 256    # graphs of the batch the autotuner times its candidates on


def batched_bench(count, steps, warmup, gen_procs=0, tune=True):
    """The batched workload (count planted-partition graphs in one CUDA-graph
    sweep loop per call) against one gsl_gsllpa call per graph; with `tune`,
    gsl_autotune_batch first picks the sweep settings on a sample of the
    graphs and the batch is timed with the defaults and with that choice."""
    import numpy as np
    import torch
    t0 = time.time()
    graphs = batched_graphs(count, gen_procs)
    gen_s = time.time() - t0
    torch.cuda.set_device(0)
    import paper_2403_01261_gb300 as gsl
    dev = torch.device("cuda", 0)
    G = len(graphs)
    off_u, col_u, vptr = pack_graphs(graphs)
    n, nnz = int(vptr[-1]), int(col_u.shape[0])
    off_d = torch.from_numpy(off_u).to(dev)
    col_d = torch.from_numpy(col_u).to(dev)
    solo = [(torch.from_numpy(o).to(dev), torch.from_numpy(c).to(dev)) for o, c in graphs]
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(ctx):
        for _ in range(warmup):
            ctx.gsllpa_batch(off_d, col_d, vptr, out=out)
        l0 = gsl.kernel_launches()
        with ClockSampler(0) as clk:
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                _, it = ctx.gsllpa_batch(off_d, col_d, vptr, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps, gsl.kernel_launches() - l0, clk.summary(), it

    base_ctx = gsl.Context(0)
    default_ms, _, _, _ = timed(base_ctx)
    default_labels = out.cpu().numpy()
    tuned = None
    ctx = base_ctx
    if tune:
        ctx = gsl.Context(0)
        ks = max(1, min(G, TUNE_SAMPLE))
        so, sc, sv = pack_graphs(graphs[:ks])
        _, tr = ctx.autotune_batch(torch.from_numpy(so).to(dev), torch.from_numpy(sc).to(dev), sv)
        tuned = {k: tr[k] for k in ("warp_max", "blk_max", "majority", "blk_threads", "blk_slots", "candidates")}
        tuned.update({"sample_graphs": ks, "sample_entry_ms": tr["entry_ms"], "sample_best_ms": tr["best_ms"]})
    batch_ms, launches, clocks, iters = timed(ctx)
    same_as_default = bool(np.array_equal(out.cpu().numpy(), default_labels))
    # per-slot device time of one batch launched directly (outside the timed region)
    ctx.set_batch_mode(False)
    ctx.set_profiling(True)
    ctx.gsllpa_batch(off_d, col_d, vptr, out=out)
    prof_direct = {p["name"]: round(p["ms"], 3) for p in ctx.profile() if p["ms"] > 0}
    ctx.set_profiling(False)
    ctx.set_batch_mode(True)
    ctx.gsllpa_batch(off_d, col_d, vptr, out=out)
    # one call per graph, graphs resident, same library
    plain = gsl.Context(0)
    outs = [torch.empty(o.numel() - 1, dtype=torch.int32, device=dev) for o, _ in solo]
    for (o, c), lab in zip(solo[:64], outs[:64]):
        plain.gsllpa(o, c, out=lab)
    torch.cuda.synchronize(dev)
    p0 = time.perf_counter()
    e0.record(stream)
    for (o, c), lab in zip(solo, outs):
        plain.gsllpa(o, c, out=lab)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = max(e0.elapsed_time(e1), (time.perf_counter() - p0) * 1e3)
    ob = out.cpu().numpy()
    same = all(np.array_equal(ob[vptr[k]:vptr[k + 1]], outs[k].cpu().numpy()) for k in range(G))
    res = {
        "value": G / (batch_ms * 1e-3), "unit": "graphs/s", "ms_per_step": batch_ms, "steps": steps,
        "warmup": warmup, "graphs": G, "n": n, "nnz": nnz,
        "plain": {"value": G / (plain_ms * 1e-3), "unit": "graphs/s", "ms": plain_ms,
                  "how": "one gsl_gsllpa call per graph, graphs resident"},
        "speedup_vs_plain": plain_ms / batch_ms, "labels_identical_to_plain": bool(same),
        "autotune": tuned, "default_setting_ms": default_ms, "tuned_gain": default_ms / batch_ms,
        "labels_identical_to_default_setting": same_as_default,
        "edges_per_s": nnz / (batch_ms * 1e-3), "max_sweeps": int(iters.max()), "mean_sweeps": float(iters.mean()),
        "gpu_launches": launches, "generation_s": gen_s, "clocks": clocks, "profile_direct_ms": prof_direct,
    }
    for c in (base_ctx, ctx, plain):
        c.close()
    return res


def run_batched(args):
    r = batched_bench(args.graphs, args.steps, args.warmup, args.gen_procs)
    line = {
        "metric": f"batched GSL-LPA graphs/s ({r['graphs']} SBM graphs, one CUDA-graph sweep loop per batch)",
        "value": r["value"], "unit": "graphs/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"batched-sbm-{r['graphs']}", "n": r["n"], "nnz": r["nnz"], "tolerance": 0.05,
                   "max_iters": 20, "mode": "sync",
                   "laws": "n log-uniform [1e3,2e5], blocks U{5..200}, degree U[8,40], ratio U[3,12]"},
        **{k: v for k, v in r.items() if k not in ("value", "ms_per_step", "steps", "warmup", "n", "nnz")},
    }
    print(json.dumps(line), flush=True)
    return 0

# ------------------------------------------------------------ compare mode
def run_compare(args):
    """Split on / off (GVE-LPA = LPA alone vs GSL-LPA = LPA + split) and the
    split techniques (union-find for Algorithm 2, Algorithm 1 with and
    without pruning) on the synthetic stand-ins: time, modularity and the
    fraction of disconnected communities (Algorithm 4)."""
    import numpy as np
    import torch
    import inputs as I
    torch.cuda.set_device(0)
    import paper_2403_01261_gb300 as gsl
    dev = torch.device("cuda", 0)
    graphs = [("sbm10k", I.sbm_planted()), ("lattice-chains", I.lattice_chains())]
    off_np, col_np = workload_graph(args.scale, args.edge_factor, args.cache, 0, 1)
    graphs.append((f"rmat{args.scale}", I.Graph(np.asarray(off_np), np.asarray(col_np))))
    ctx = gsl.Context(0)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return r, statistics.median(ms)

    rows = []
    for name, g in graphs:
        off = torch.from_numpy(g.offsets).to(dev)
        col = torch.from_numpy(g.cols).to(dev)
        lab, gve_ms = timed(lambda: ctx.lpa(off, col, tolerance=0.05, max_iters=20))
        out, gsl_ms = timed(lambda: ctx.gsllpa(off, col, tolerance=0.05, max_iters=20))
        out_a, async_ms = timed(lambda: ctx.gsllpa(off, col, tolerance=0.05, max_iters=20, mode=1))
        (_, k_uf), uf_ms = timed(lambda: ctx.split(off, col, lab))
        (_, lp_sweeps), lp_ms = timed(lambda: ctx.split_lp(off, col, lab, pruning=False), reps=1)
        (_, lpp_sweeps), lpp_ms = timed(lambda: ctx.split_lp(off, col, lab, pruning=True), reps=1)
        comms = int(torch.unique(lab).numel())
        disc = ctx.disconnected(off, col, lab)
        rows.append({
            "graph": name, "n": g.n, "nnz": g.nnz,
            "gve_lpa": {"ms": gve_ms, "modularity": ctx.modularity(off, col, lab), "communities": comms,
                        "disconnected": disc, "disconnected_fraction": disc / max(1, comms)},
            "gsl_lpa": {"ms": gsl_ms, "modularity": ctx.modularity(off, col, out), "communities": k_uf,
                        "disconnected": ctx.disconnected(off, col, out)},
            "gsl_lpa_async": {"ms": async_ms, "modularity": ctx.modularity(off, col, out_a),
                              "communities": int(torch.unique(out_a).numel()),
                              "disconnected": ctx.disconnected(off, col, out_a)},
            "split_ms": {"union_find": uf_ms, "sl_lp": lp_ms, "sl_lpp": lpp_ms},
            "split_sweeps": {"sl_lp": lp_sweeps, "sl_lpp": lpp_sweeps},
        })
        del off, col
    line = {"metric": "GVE-LPA vs GSL-LPA (split on/off) and split techniques on the synthetic stand-ins",
            "unit": "ms", "n_gpus": 1, "data": "synthetic", "dtype": "int32", "higher_is_better": False,
            "config": {"workload": "compare", "tolerance": 0.05, "max_iters": 20, "mode": "sync"}, "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- served mode
def _gen_served(ks):
    import inputs as I
    out = []
    for k in ks:
        g = I.served_request(k, threads=1)
        out.append((k, g.offsets, g.cols))
    return out


def served_pool(count, procs):
    """Request graphs 0..count-1 of the served workload (inputs.served_request)."""
    import multiprocessing as mp
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    chunks = [list(range(p, count, procs)) for p in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_gen_served, chunks)
    got = sorted((x for part in parts for x in part), key=lambda x: x[0])
    return [(o, c) for _, o, c in got]


def _serve_at(srv, pool, rate, duration, seed):
    """Poisson arrivals at `rate` for `duration` s, each a random pool graph;
    returns per-request (pool index, request info, labels of the first few)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 16)
    times = np.cumsum(gaps)
    times = times[times < duration]
    picks = rng.integers(0, len(pool), size=len(times))
    ids = [None] * len(times)
    submitted = threading.Event()
    t_start = time.perf_counter()

    def submitter():
        for i, (t, k) in enumerate(zip(times, picks)):
            delay = t_start + t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids[i] = srv.submit(*pool[k])
        submitted.set()

    th = threading.Thread(target=submitter, daemon=True)
    th.start()
    infos, labels = [], {}
    for i in range(len(times)):
        while ids[i] is None:
            time.sleep(0.0002)
        lab, info = srv.wait(ids[i], info=True)
        infos.append(info)
        if int(picks[i]) not in labels:
            labels[int(picks[i])] = lab.copy()
    t_end = time.perf_counter()
    th.join()
    return picks, infos, labels, t_end - t_start


def served_bench(pool_size, rate, duration, slots, gen_procs=0):
    """Served workload: Poisson arrivals of request graphs (70 % planted
    partition, 30 % R-MAT, n log-uniform 1e3..2^22) drawn from a pinned host
    pool of pool_size distinct graphs, through the library's
    continuous-batching server, at the offered rate and at half the achieved
    rate; against one gsl_gsllpa_host call per request, one at a time."""
    import numpy as np
    import torch
    t0 = time.time()
    raw = served_pool(pool_size, gen_procs)
    gen_s = time.time() - t0
    torch.cuda.set_device(0)
    import paper_2403_01261_gb300 as gsl
    pool, keep = [], []
    for o, c in raw:
        to, tc = torch.from_numpy(o).pin_memory(), torch.from_numpy(c).pin_memory()
        keep.append((to, tc))
        pool.append((to.numpy(), tc.numpy()))
    del raw
    # plain: one request at a time through the host-buffer entry point
    ctx = gsl.Context(0)
    outs = [torch.empty(o.shape[0] - 1, dtype=torch.int32).pin_memory() for o, _ in pool]
    for (o, c), lab in list(zip(keep, outs))[:4]:
        ctx.gsllpa_host(o, c, out=lab)
    p0 = time.perf_counter()
    for (o, c), lab in zip(keep, outs):
        ctx.gsllpa_host(o, c, out=lab)
    plain_s = time.perf_counter() - p0
    plain_gps = len(pool) / plain_s
    ctx.close()
    srv = gsl.Server(device=0, slots=slots, memory_fraction=0.6, tolerance=0.05, max_iters=20)
    for k in range(min(4, len(pool))):     # warm-up
        srv.wait(srv.submit(*pool[k]))
    runs = []
    launches0 = gsl.kernel_launches()
    clocks = []
    for rate_k in (rate, None):
        if rate_k is None:   # a second, lighter load where p99 is not queueing-dominated
            rate_k = 0.5 * min(rate, runs[0]["achieved_rps"])
        with ClockSampler(0) as clk:
            picks, infos, labels, wall = _serve_at(srv, pool, rate_k, duration, seed=len(runs))
        clocks.append(clk.summary())
        lat = np.array([i["latency_ms"] for i in infos])
        que = np.array([i["queue_ms"] for i in infos])
        svc = np.array([i["service_ms"] for i in infos])
        dev = {k: np.array([i[k] for i in infos]) for k in ("h2d_ms", "compute_ms", "d2h_ms")}
        runs.append({"offered_rps": rate_k, "requests": len(infos), "achieved_rps": len(infos) / wall,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "queue_p50_ms": float(np.percentile(que, 50)), "service_p50_ms": float(np.percentile(svc, 50)),
                     "service_mean_ms": float(svc.mean()),
                     "device_mean_ms": {k: float(v.mean()) for k, v in dev.items()},
                     "mean_batch_graphs": float(np.mean([i["batch_graphs"] for i in infos])),
                     "same_as_plain": all(np.array_equal(lab, outs[k].numpy()) for k, lab in labels.items())})
    launches = gsl.kernel_launches() - launches0
    st = srv.stats()
    srv.close()
    nnz = np.array([c.shape[0] for _, c in pool])
    return {
        "value": runs[0]["achieved_rps"], "unit": "graphs/s", "rate_rps": rate, "duration_s": duration,
        "pool": len(pool), "slots": slots, "mean_nnz": float(nnz.mean()),
        "p50_ms": runs[0]["p50_ms"], "p99_ms": runs[0]["p99_ms"], "runs": runs,
        "plain": {"value": plain_gps, "unit": "graphs/s", "how": "one gsl_gsllpa_host call per pool graph, pinned"},
        "speedup_vs_plain": runs[0]["achieved_rps"] / plain_gps,
        "max_possible_speedup_at_rate": rate / plain_gps,
        "labels_identical_to_plain": all(r["same_as_plain"] for r in runs),
        "server": st, "gpu_launches": launches, "generation_s": gen_s, "clocks": clocks,
        "e2e": {"value": runs[0]["achieved_rps"], "unit": "graphs/s",
                "h2d_bytes_per_step": int(8 * sum(o.shape[0] for o, _ in pool) + 4 * nnz.sum()) // len(pool),
                "d2h_bytes_per_step": int(4 * sum(o.shape[0] - 1 for o, _ in pool)) // len(pool)},
    }


def run_served(args):
    r = served_bench(args.pool, args.rate, args.duration, args.slots, args.gen_procs)
    line = {
        "metric": "served GSL-LPA graphs/s with p50/p99 latency (Poisson arrivals, continuous batching)",
        "value": r["value"], "unit": "graphs/s", "n_gpus": 1, "steps": len(r["runs"]), "warmup": 4,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"served-pool{r['pool']}", "rate_rps": args.rate, "duration_s": args.duration,
                   "slots": args.slots, "mix": "70% planted partition / 30% R-MAT ef16, n log-uniform 1e3..2^22",
                   "mean_nnz": r["mean_nnz"], "tolerance": 0.05, "max_iters": 20, "mode": "sync"},
        **{k: v for k, v in r.items() if k not in ("value", "rate_rps", "duration_s", "pool", "slots", "mean_nnz")},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU side
def dominant_roofline(profile, peaks):
    slots = [s for s in profile if s["ms"] > 0 and s["bytes"] > 0]
    if not slots:
        return None
    top = max(slots, key=lambda s: s["ms"])
    achieved = top["bytes"] / (top["ms"] * 1e-3) / 1e9
    peak, src = peaks
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            from paper_2403_01261_gb300 import _build
            rec = json.load(open(tpath))
            if rec.get("source_hash") == _build.source_hash() and top["name"] in rec.get("per_launch", {}):
                traffic = rec["per_launch"][top["name"]]
        except Exception:  # noqa: BLE001
            traffic = None
    return {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": src,
            "bytes_per_launch": top["bytes"] / max(1, top["launches"]),
            "ms_per_launch": top["ms"] / max(1, top["launches"]), "launches": top["launches"]}


SPLIT_SLOTS = ("split_unionfind", "split_count_renumber")


def phase_roofline(profile, peak, steps, step_ms):
    """Algorithmic bytes over device time for the whole sweep phase (every
    slot but the split and modularity) and for the whole step (every slot's
    bytes over the measured step time)."""
    sweep = [s for s in profile if s["name"] not in SPLIT_SLOTS and s["name"] != "modularity"]
    sb = sum(s["bytes"] for s in sweep)
    sms = sum(s["ms"] for s in sweep)
    tb = sum(s["bytes"] for s in profile if s["name"] != "modularity")
    out = {}
    if sms > 0:
        a = sb / (sms * 1e-3) / 1e9
        out["sweep_phase"] = {"achieved": a, "frac": a / peak, "bytes_per_step": sb / steps,
                              "ms_per_step": sms / steps}
    if step_ms > 0:
        a = tb / steps / (step_ms * 1e-3) / 1e9
        out["step"] = {"achieved": a, "frac": a / peak, "bytes_per_step": tb / steps, "ms_per_step": step_ms}
    return out


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except Exception:  # noqa: BLE001
            pass
    return 6800.0, "fallback"


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "compare":
        return run_compare(args)
    import numpy as np
    import torch
    rank, world, local = rank_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    import paper_2403_01261_gb300 as gsl

    offsets_np, cols_np = workload_graph(args.scale, args.edge_factor, args.cache, rank, world)
    n = offsets_np.shape[0] - 1
    nnz = cols_np.shape[0]
    dev = torch.device("cuda", local)
    off_h = torch.from_numpy(np.ascontiguousarray(offsets_np)).pin_memory()
    col_h = torch.from_numpy(np.ascontiguousarray(cols_np)).pin_memory()
    off = off_h.to(dev)
    col = col_h.to(dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    ctx = gsl.Context(local)
    mode = 1 if args.mode == "async" else 0
    stream = torch.cuda.current_stream(dev)
    wt = edge_weights(off, col, args.weights) if args.weights != "unit" else None
    if args.weights == "f32":
        def step(**kw):
            return ctx.gsllpa_f32(off, col, wt, tolerance=0.05, max_iters=20, mode=mode, out=out, **kw)
    else:
        def step(**kw):
            return ctx.gsllpa(off, col, wt, tolerance=0.05, max_iters=20, mode=mode, out=out, **kw)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # timed region: K steps on resident inputs (cols >> L2, so no flush needed)
    ctx.set_profiling(True)
    stats = []
    launches0 = gsl.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            _, st = step(stats=True)
            stats.append(st)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    launches = gsl.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = ctx.profile()
    ctx.set_profiling(False)
    ms = max_over_ranks(ms, world, dev)

    # end to end through the host-buffer entry point (copies inside the region)
    e2e = None
    if not args.no_e2e and args.weights == "unit":
        lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
        ctx.gsllpa_host(off_h, col_h, tolerance=0.05, max_iters=20, mode=mode, out=lab_h)   # warm the staging
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            ctx.gsllpa_host(off_h, col_h, tolerance=0.05, max_iters=20, mode=mode, out=lab_h)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        wall = (time.perf_counter() - t0) / args.e2e_steps
        e2e_ms = max(e0.elapsed_time(e1) / args.e2e_steps, wall * 1e3)
        e2e_ms = max_over_ranks(e2e_ms, world, dev)
        e2e = {"value": replicas_value(world, nnz, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": 8 * (n + 1) + 4 * nnz,
               "d2h_bytes_per_step": 4 * n, "ms_per_step": e2e_ms}
        if mode == 0:
            assert torch.equal(lab_h, out.cpu()), "host-buffer path disagrees with the device path"

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    st = stats[-1]
    T = st["iterations"]
    lpa_ms = statistics.median(s["ms_lpa"] for s in stats)
    split_ms = statistics.median(s["ms_split"] for s in stats)
    peak = hbm_peak()
    roof = dominant_roofline(prof, peak)
    if roof:
        roof.update(phase_roofline(prof, peak[0], args.steps, ms))
    clocks = clk.summary()
    gpu_labels = out.cpu().numpy()
    del ctx, off, col, out, wt
    torch.cuda.empty_cache()
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(offsets_np, cols_np, 0.05, 20, f"R-MAT scale {args.scale} ef {args.edge_factor}",
                           gpu_labels if args.weights == "unit" and mode == 0 else None, st["changed"])
        cpu.pop("seconds", None)
    extra = {}
    if world == 1 and not args.no_batched:
        extra["batched"] = batched_bench(args.graphs, 3, 2, args.gen_procs)
    if world == 1 and not args.no_served:
        extra["served"] = served_bench(args.pool, args.rate, args.line_served_duration, args.slots,
                                       args.gen_procs)
    line = {
        "metric": METRIC, "value": replicas_value(world, nnz, ms), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 weights, f64 sums" if args.weights == "f32" else "int32", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale}-ef{args.edge_factor}", "rmat_abcd": [0.57, 0.19, 0.19, 0.05],
                   "n": n, "nnz": nnz, "tolerance": 0.05, "max_iters": 20, "mode": args.mode, "seed": 1,
                   "weights": args.weights,
                   "parallelism": f"replicas{world}", "l2": f"inputs larger than L2 (cols {4 * nnz / 1e9:.2f} GB)"},
        "sweeps": T, "communities": st["communities"], "lpa_ms": lpa_ms, "split_ms": split_ms,
        "edges_iter_per_s": world * nnz * T / (ms * 1e-3),
        "edges_scanned_per_s": world * st["edges_scanned"] / (ms * 1e-3),
        "changed": st["changed"], "active": st["active"],
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        **extra,
    }
    if args.profile_json:
        with open(args.profile_json, "w") as f:
            json.dump({"profile": prof, "steps": args.steps, "line": line}, f, indent=1)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
