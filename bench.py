#!/usr/bin/env python
"""PCPM PageRank benchmark: per-iteration GTEPS on one GB300 (or N destination shards).

Workload (default): RMAT scale 24 (16,777,216 nodes), edge factor 16,
a, b, c = 0.57, 0.19, 0.19, random node labels, duplicates and self-loops
removed, uint32 CSR, partition size 32,768 nodes (k = 512), d = 0.85, FP32
ranks with FP64 reductions. A step is one PCPM iteration: scatter, gather +
apply, reduce. Inputs (about 3 GB per iteration) are far larger than the
129 MB L2, so no flush is needed between steps.

Prints one JSON line. `value` = edges / (device time of one iteration) in
GTEPS, from CUDA events recorded by the library on the launching stream;
`roofline` covers the kernel with the largest share of the time; `other_mode`
times the other iteration form (fused gather + next scatter); `e2e` is the
same metric through the host-memory entry point pcpm_pagerank_host (H2D copy
of the CSR from pinned memory, PNG build, 20 iterations, D2H of the ranks);
`cpu_baseline` times the FP64 CPU oracle on the host on one full iteration of
the same graph. `--impl reference` times only the oracle (rank 0), each step a
bounded slice of that iteration.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS per iter & achieved HBM GB/s; time to L1 residual 1e-7 vs plain FP32"
PHASES = ("scatter", "gather_apply", "reduce")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400, help="timed iterations")
    ap.add_argument("--warmup", type=int, default=5, help="untimed iterations before timing (>= 3)")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--graph", choices=("rmat", "er"), default="rmat")
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--edge-factor", type=float, default=16.0)
    ap.add_argument("--labels", choices=("random", "bfs"), default="random")
    ap.add_argument("--part-size", type=int, default=32768)
    ap.add_argument("--d", type=float, default=0.85)
    ap.add_argument("--seed", type=int, default=1710)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-converge", action="store_true", help="skip the time-to-residual run")
    ap.add_argument("--no-two-phase", action="store_true", help="skip the two-phase (per-phase) leg")
    ap.add_argument("--no-update-dtypes", action="store_true", help="skip the 16-bit update-bin leg")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned warm start (trained on 64 RMAT graphs, scales 18-22, a in "
                         "[0.45, 0.65]; iterations and time to residual 1e-7 against the uniform start)")
    ap.add_argument("--ws-graphs", type=int, default=64, help="training graphs of the warm-start leg")
    ap.add_argument("--no-spmv", action="store_true", help="skip the weighted SpMV leg")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 256 RMAT graphs of scales 10-18 solved by one captured CUDA graph launch")
    ap.add_argument("--no-ppr", action="store_true",
                    help="skip batched personalized PageRank: RMAT s22, 64 teleport columns, 20 iterations")
    ap.add_argument("--ppr-scale", type=int, default=22, help="RMAT scale of the --ppr leg (22: the batched workload)")
    ap.add_argument("--mode", choices=("fused", "two_phase"), default="two_phase",
                    help="iteration form timed for `value` (the other is reported in other_mode)")
    ap.add_argument("--gather-layout", choices=("windows", "chunks"), default="windows",
                    help="gather copy of the IDs: owner windows without atomics (default) or 256-ID chunks with "
                         "shared-memory atomics")
    ap.add_argument("--ref-budget-s", type=float, default=120.0, help="reference arm: timed seconds target")
    return ap.parse_args()


def workload_name(a):
    if a.graph == "rmat":
        g = f"rmat-s{a.scale}-ef{a.edge_factor:g}-abc0.57/0.19/0.19"
    else:
        g = f"er-n{1 << a.scale}-deg{a.edge_factor:g}"
    return f"{g}-{a.labels}-labels-q{a.part_size}"


def make_graph(a):
    import graphgen
    if a.graph == "rmat":
        return graphgen.rmat(a.scale, a.edge_factor, 0.57, 0.19, 0.19, seed=a.seed, relabel=a.labels)
    return graphgen.erdos_renyi(1 << a.scale, a.edge_factor, seed=a.seed, relabel=a.labels)


def layout_option(a):
    """The build option gather_windows for --gather-layout."""
    return 2 if a.gather_layout == "chunks" else 0


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class Replicas:
    """The N ranks of one node, each running an independent replica of the
    whole job (the path has no exchange step, so no data-path collective):
    a barrier around the timed region and the maximum of a per-rank time.
    NCCL on GPUs; gloo with device "cpu" runs the same logic on host ranks."""

    def __init__(self, backend: str = "nccl", device=None):
        self.rank, self.world, self.local = dist_env()
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            kw = {"device_id": torch.device(device)} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def aggregate_gteps(self, edges_per_replica: int, slowest_seconds_per_step: float) -> float:
        """Whole-job GTEPS: the edges all replicas processed in one step over
        the slowest rank's step time (the value `max` returned)."""
        return self.world * edges_per_replica / slowest_seconds_per_step / 1e9

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle sampling in the background (read-only)."""

    FIELDS = ("index,timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[1].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    frac = float("0." + parts[1].split(".")[1]) if "." in parts[1] else 0.0
                    rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[6:10]))
                except (ValueError, IndexError):
                    continue
        os.unlink(self.path)
        inside = [r for r in rows if t0 - 0.06 <= r[0] <= t1 + 0.06]
        used = inside or rows
        if not used:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in used for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in used), "sm_max_mhz": max(r[2] for r in used),
                "reasons": reasons, "samples": len(used), "samples_in_timed_region": len(inside)}


# --------------------------------------------------------------- roofline
def algorithmic_bytes(info, mode="fused"):
    """Bytes each kernel must move per launch (4-byte indices and ranks;
    updates of info["update_bytes"], 4 unless the bins are 16-bit)."""
    n, m, ne, k = info["n"], info["num_edges"], info["num_updates"], info["num_partitions"]
    ub = info.get("update_bytes", 4)
    if info.get("gather_windows"):
        # destIDs, updates, window headers (64 B) and descriptors (16 B), bins, hubs
        gather = 4 * m + ub * ne + 80 * info["num_windows"] + 8 * (k + 1) + 4 * 8 * k
    else:
        nchunks = -(-m // 256)
        gather = 4 * m + ub * ne + 4 * nchunks + 8 * (k + 1) + 8 * k  # destIDs, updates, chunk bases, bins, hubs
    apply = 12 * n  # PR_old and 1/outdeg read, PR' written
    if mode == "fused":
        # the fused gather's scatter reads 4-byte global source IDs
        scatter = (4 + ub) * ne + 8 * k * k  # srcIdx read + update write, segment starts/counts
        return {"scatter": 0, "gather_apply": gather + apply + scatter, "reduce": 16 * k}
    # the scatter kernel reads 2-byte local source indices (u - p q) with
    # FP32 bins, 4-byte global ones with 16-bit bins
    scatter = ((2 if ub == 4 else 4) + ub) * ne + 8 * k * k
    return {"scatter": scatter + 8 * n, "gather_apply": gather + apply, "reduce": 16 * k}


def eq5_bytes(info):
    """The paper's PCPM communication model, Eq. 5, with d_i = d_v = 4."""
    n, m, ne, k = info["n"], info["num_edges"], info["num_updates"], info["num_partitions"]
    r = m / ne if ne else 1.0
    return m * (4 * (1 + 1 / r) + 8 / r) + k * k * 4 + 2 * n * 4


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(kernel: str, layout: str, algorithmic: int):
    """DRAM bytes per launch of `kernel`: the ratio of DRAM bytes to
    algorithmic bytes from a committed single-kernel ncu capture (on a smaller
    graph of the same family, profiles/traffic.json) times this workload's
    algorithmic bytes. None unless the kernel sources are unchanged since the
    capture and the capture is of the same gather layout."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        rec = json.load(f)
    for name, sha in rec.get("source_sha256", {}).items():
        src = os.path.join(ROOT, "paper_1709_07122_gb300", "csrc", name)
        if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != sha:
            return None, None
    entry = rec.get("kernels", {}).get(kernel)
    if not entry or entry.get("layout") != layout:
        return None, None
    ratio = entry["dram_bytes"] / entry["algorithmic_bytes"]
    note = "ncu DRAM/algorithmic ratio %.3f from a single-kernel capture on %s, times this workload's " \
           "algorithmic bytes" % (ratio, entry["capture_workload"])
    return int(round(ratio * algorithmic)), note


# ---------------------------------------------------------------- CPU side
def cpu_oracle_baseline(rp, col, d, tol=1e-7, max_iters=100):
    """The FP64 oracle on the host: one full pull iteration (Eq. 1) from the
    uniform start on all host threads and on one thread, then the threaded
    iteration run to L1 change `tol`. Returns (cpu_baseline dict, first
    iteration's vector)."""
    import oracle
    pull = oracle.Pull(rp, col)
    n, m = pull.n, int(rp[-1])
    threads = oracle.host_threads()
    x = np.full(n, 1.0 / n)
    y = np.empty(n)
    t0 = time.perf_counter()
    pull.step_all(x, y, d, threads=threads)
    dt_mt = time.perf_counter() - t0
    y1 = y.copy()
    t0 = time.perf_counter()
    pull.step_all(x, y, d, threads=1)
    dt_1 = time.perf_counter() - t0
    xs, ys = x.copy(), np.empty(n)
    iters, r = 0, float("inf")
    t0 = time.perf_counter()
    while r >= tol and iters < max_iters:
        r = pull.step_all(xs, ys, d, threads=threads)
        xs, ys = ys, xs
        iters += 1
    dt_res = time.perf_counter() - t0
    out = {"value": m / dt_mt / 1e9, "unit": "GTEPS", "cores": threads, "kind": "oracle",
           "sample": "one full FP64 pull iteration (Eq. 1) of the same graph from the uniform start, %.2f s on %d "
                     "host threads (contiguous destination ranges)" % (dt_mt, threads),
           "single_thread": {"value": m / dt_1 / 1e9, "unit": "GTEPS", "cores": 1, "seconds": dt_1},
           "time_to_residual": {"tol": tol, "iters": iters, "seconds": dt_res, "reached": r < tol,
                                "final_residual": r, "cores": threads}}
    return out, y1


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    if a.warmup < 0 or a.steps < 1:
        raise SystemExit("steps must be >= 1")
    rp, col = make_graph(a)
    n, m = rp.size - 1, int(rp[-1])
    pull = oracle.Pull(rp, col)
    threads = oracle.host_threads()
    x = np.full(n, 1.0 / n)
    y = np.empty(n)
    dmass = pull.dangling_mass(x)
    # Size each step so the whole run stays near the time budget.
    probe = max(1, n // 256)
    t0 = time.perf_counter()
    pull.step_all(x, y, a.d, threads=threads, v_begin=0, v_end=probe, dmass=dmass)
    per_edge = (time.perf_counter() - t0) / max(1, pull.in_edges(0, probe))
    budget_edges = a.ref_budget_s / max(per_edge, 1e-12) / (a.steps + a.warmup)
    width = int(min(n, max(1024, budget_edges / max(m / n, 1e-9))))
    starts = [(i * width) % n for i in range(a.steps + a.warmup)]
    for s in starts[:a.warmup]:
        pull.step_all(x, y, a.d, threads=threads, v_begin=s, v_end=min(n, s + width), dmass=dmass)
    edges = 0
    t0 = time.perf_counter()
    for s in starts[a.warmup:]:
        e = min(n, s + width)
        pull.step_all(x, y, a.d, threads=threads, v_begin=s, v_end=e, dmass=dmass)
        edges += pull.in_edges(s, e)
    dt = time.perf_counter() - t0
    gteps = edges / dt / 1e9
    sample = (f"FP64 pull step (Eq. 1) of the oracle over {a.steps} slices of {width} destination nodes "
              f"of the full graph ({edges} in-edges in total), {threads} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": gteps, "unit": "GTEPS", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3 / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": n, "m": m, "part_size": a.part_size, "d": a.d},
        "cpu_baseline": {"value": gteps, "unit": "GTEPS", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": gteps, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU side
def spmv_leg(a, rp, col, m):
    """Weighted SpMV y = A^T_w x over the PNG (Sec. 3.5) on the same graph:
    random weights, q = 16384 (the weighted gather's limit), GTEPS of the
    product (scatter of x + weighted gather) from CUDA events."""
    import torch
    import paper_1709_07122_gb300 as pcpm
    q = min(a.part_size, 16384)
    rng = np.random.default_rng(a.seed + 11)
    w = torch.from_numpy(rng.random(m, dtype=np.float32)).cuda()
    x = torch.from_numpy(rng.random(rp.size - 1, dtype=np.float32)).cuda()
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    res = {}
    with pcpm.PNG.weighted(d_rp, d_col, w, q) as gw, pcpm.PNG(d_rp, d_col, q) as gu:
        for name, g in (("weighted", gw), ("unit_weights", gu)):
            y = torch.empty_like(x)
            for _ in range(3):
                g.spmv(x, y)
            reps = 20
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                g.spmv(x, y)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[name] = {"ms": ms, "gteps": m / (ms * 1e-3) / 1e9}
    # a non-square matrix: the first half of the rows, all columns (Sec. 3.5)
    rows = (rp.size - 1) // 2
    mr = int(rp[rows])
    r_rp, r_col = pcpm.to_device_csr(rp[:rows + 1], col[:mr])
    xr = torch.from_numpy(rng.random(rows, dtype=np.float32)).cuda()
    with pcpm.PNG.rect(r_rp, r_col, rp.size - 1, q, w[:mr].contiguous()) as gr:
        for _ in range(3):
            gr.spmv_rect(xr)
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            gr.spmv_rect(xr)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res["rect_weighted"] = {"rows": rows, "cols": rp.size - 1, "entries": mr, "ms": ms,
                                "gteps": mr / (ms * 1e-3) / 1e9}
    del d_rp, d_col, w, x, r_rp, r_col, xr
    torch.cuda.empty_cache()
    res["part_size"] = q
    res["note"] = "one scatter of x (no 1/outdeg) + one gather; weighted stages 4 extra bytes per edge"
    return res


def ppr_leg(a, iters: int = 20):
    """Batched personalized PageRank (pcpm_ppr_*): RMAT scale 22 (--ppr-scale; random labels,
    q = 32768), 64 teleport columns each uniform over 1-1000 random seed nodes,
    `iters` iterations from R = T, timed with CUDA events on the stream. Against
    it: the same graph's single-vector PageRank iteration, times 64."""
    import torch
    import graphgen
    import paper_1709_07122_gb300 as pcpm
    rp, col = graphgen.rmat(a.ppr_scale, a.edge_factor, 0.57, 0.19, 0.19, seed=a.seed + 22, relabel="random")
    n, m = rp.size - 1, int(rp[-1])
    rng = np.random.default_rng(a.seed + 23)
    ptr, idx = [0], []
    for _ in range(pcpm.PPR_COLS):
        k = int(rng.integers(1, 1001))
        idx.extend(rng.choice(n, size=k, replace=False).tolist())
        ptr.append(len(idx))
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    with pcpm.PNG(d_rp, d_col, 32768) as g:
        info = g.info
        ne = info["num_updates"]
        g.iterate(a.d, 3, mode="two_phase")
        single = g.iterate_timed(a.d, 10, mode="two_phase")["span"] / 10  # ms per iteration
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        p = pcpm.PPR(g, np.array(ptr, np.uint32), np.array(idx, np.uint32))
        create_ms = (time.perf_counter() - c0) * 1e3
        with p:
            p.run(a.d, 3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            p.run(a.d, iters)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / iters
            res = p.residuals()
            pinfo = p.info
    del d_rp, d_col
    torch.cuda.empty_cache()
    row = 4 * pcpm.PPR_COLS
    # scatter: R rows read, update rows written, positions; gather: update
    # rows read once, entry index, R_old read, R' written
    alg = n * row + ne * row + 4 * ne + 4 * (n + 1) + ne * row + 4 * m + 4 * (n + 1) + 2 * n * row
    peak, src = measured_peaks()
    return {"workload": "rmat-s%d-ef%g-random-labels-q32768, 64 teleport columns (1-1000 seeds each)"
                        % (a.ppr_scale, a.edge_factor),
            "n": n, "m": m, "num_updates": ne, "iters": iters, "ms_per_iter": ms,
            "gteps_x64": m * pcpm.PPR_COLS / (ms * 1e-3) / 1e9,
            "single_vector_ms_per_iter": single,
            "speedup_vs_64_single_vector_iterations": 64 * single / ms,
            "algorithmic_bytes_per_iter": alg,
            "hbm_frac_of_%s" % src: alg / (ms * 1e-3) / 1e9 / peak,
            "split_destinations": pinfo["split_destinations"], "create_ms": create_ms,
            "last_l1_change_max_over_columns": float(res[-1].max())}


def batched_leg(a, graphs: int = 256, iters: int = 20):
    """Many small independent graphs (RMAT, scales drawn from 10-18, random
    labels) solved for `iters` iterations each by one captured CUDA graph
    launch, against the same solves issued call by call on one stream.
    Graphs that share a part size and cluster size run each phase as one
    launch over all their units, so the configuration is tuned for the batch
    as a whole: one part size for every graph (2048, 8192 or 32768, default
    tiles), or part size and tile shape per scale as the single-graph
    autotuner picks them (five timed iterations on the first graph of that
    scale), or each graph's node count rounded into [2048, 32768] (one
    partition per graph up to scale 15). The fastest configuration is the
    leg's number."""
    import torch
    import paper_1709_07122_gb300 as pcpm
    import graphgen
    rng = np.random.default_rng(a.seed + 21)
    scales = [int(s) for s in rng.integers(10, 19, size=graphs)]
    t0 = time.perf_counter()
    data = [graphgen.rmat(s, a.edge_factor, seed=a.seed + 3000 + i, relabel="random") for i, s in enumerate(scales)]
    gen_s = time.perf_counter() - t0
    dev = [pcpm.to_device_csr(rp, col) for rp, col in data]
    edges = sum(int(rp[-1]) for rp, _ in data)

    def time_batch(batch):
        batch.launch()
        torch.cuda.synchronize()
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.launch()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    # part size and tile shape per scale (pcpm_autotune_ex on the first graph
    # of that scale)
    best_q, best_opts = {}, {}
    shapes = ({}, {"gather_cluster": 1}, {"gather_unit_chunks": 64})
    for s in sorted(set(scales)):
        i = scales.index(s)
        best_q[s], best_opts[s], _ = pcpm.autotune_tiles(*dev[i], (2048, 8192, 32768), shapes, a.d, warmup=2,
                                                         iters=5, mode="two_phase")
    configs = {"part_size_%d" % q: [(q, {})] * graphs for q in (2048, 8192, 32768)}
    # each graph in one partition where it fits: n = 2^scale rounded into
    # [2048, 32768], so small graphs' CTAs reserve small accumulators
    configs["part_size_fit"] = [(min(32768, max(2048, 1 << s)), {}) for s in scales]
    configs["per_scale_autotuned"] = [(best_q[s], best_opts[s]) for s in scales]
    results, best = {}, None
    for name, cfg in configs.items():
        handles = [pcpm.PNG(*dev[i], q, **opts) for i, (q, opts) in enumerate(cfg)]
        t1 = time.perf_counter()
        batch = pcpm.Batch(handles, a.d, iters, mode="two_phase")
        capture_ms = (time.perf_counter() - t1) * 1e3
        ms = time_batch(batch)
        results[name] = {"ms": ms, "gteps": edges * iters / (ms * 1e-3) / 1e9,
                         "kernel_launches": batch.kernel_launches, "capture_ms": capture_ms}
        if best is None or ms < results[best[0]]["ms"]:
            if best is not None:
                best[1].close()
                for h in best[2]:
                    h.close()
            best = (name, batch, handles)
        else:
            batch.close()
            for h in handles:
                h.close()
    del dev
    name, batch, handles = best
    # the same work, one call after another
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for h in handles:
        h.reset()
        h.iterate(a.d, iters, sync=False, mode="two_phase")
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    batch.close()
    # equal accuracy: the fewest iterations after which every graph's L1
    # change is below 1e-7 (read from one long batch), then that batch timed
    tol, long_iters = 1e-7, 80
    with pcpm.Batch(handles, a.d, long_iters, mode="two_phase") as lb:
        lb.launch()
        torch.cuda.synchronize()
        need = []
        for h in handles:
            hist = h.residual_history()
            below = np.nonzero(hist < tol)[0]
            need.append(int(below[0]) + 1 if below.size else None)
    to_tol = {"tol": tol, "reached": all(x is not None for x in need)}
    if to_tol["reached"]:
        k_tol = max(need)
        with pcpm.Batch(handles, a.d, k_tol, mode="two_phase") as tb:
            to_tol.update({"iters": k_tol, "ms": time_batch(tb),
                           "iters_per_graph_min_median_max": [min(need), int(np.median(need)), k_tol]})
    for h in handles:
        h.close()
    r = results[name]
    return {"graphs": graphs, "scales": "10-18", "iterations_each": iters, "edges_total": edges,
            "time_to_residual": to_tol,
            "config": name, "one_graph_launch_ms": r["ms"], "gteps": r["gteps"],
            "kernel_launches": r["kernel_launches"], "configs": results,
            "per_scale_autotuned": {"partition_size": {str(k): v for k, v in sorted(best_q.items())},
                                    "tile_shape": {str(k): v for k, v in sorted(best_opts.items())}},
            "call_by_call_ms": seq_ms, "call_by_call_gteps": edges * iters / (seq_ms * 1e-3) / 1e9,
            "generate_s": gen_s}


def warm_start_leg(a, rp, col):
    """Learned warm start (not in the paper): train on RMAT graphs of scales
    18-22 with a drawn from [0.45, 0.65], then solve the benchmark graph (not
    among them) to L1 residual 1e-7 from the uniform and from the warm start."""
    import torch
    from paper_1709_07122_gb300 import warmstart as ws
    import graphgen
    rng = np.random.default_rng(a.seed + 7)
    t0 = time.perf_counter()
    samples, shapes = [], []
    for i in range(a.ws_graphs):
        s, aa = int(rng.integers(18, 23)), float(rng.uniform(0.45, 0.65))
        trp, tcol = graphgen.rmat(s, a.edge_factor, *ws.rmat_params(aa), seed=a.seed + 1000 + i, relabel="random")
        samples.append(ws.Sample(trp, tcol, a.part_size, a.d))
        shapes.append((s, round(aa, 3)))
        del trp, tcol
    data_s = time.perf_counter() - t0
    params = ws.init_params(samples, seed=a.seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    log = ws.train(params, samples, steps=1500, batch=65536, lr=3e-3, log_every=250, schedule="cosine")
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    nodes = sum(s.n for s in samples)
    del samples
    torch.cuda.empty_cache()
    res = ws.evaluate(params, rp, col, a.part_size, a.d, tol=1e-7)
    diff = float((res["warm"]["ranks"] - res["uniform"]["ranks"]).abs().sum())
    return {"train_graphs": len(shapes), "train_nodes": nodes, "scales": sorted({s for s, _ in shapes}),
            "data_seconds": data_s, "train_seconds": train_s, "steps": 1500, "batch": 65536,
            "lr": "3e-3, cosine decay",
            "loss_log": log, "tol": 1e-7,
            "uniform": {k: res["uniform"][k] for k in ("iters", "ms", "residual")},
            "warm": {k: res["warm"][k] for k in ("iters", "ms", "residual")},
            "warm_ms_includes": "features (incl. one PCPM iteration), inference, softmax",
            "l1_between_final_ranks": diff}


def run_ours(a):
    import torch
    import paper_1709_07122_gb300 as pcpm

    rank, world, local = dist_env()
    if a.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    torch.cuda.set_device(local)
    ranks = Replicas("nccl", f"cuda:{local}")
    barrier, max_over_ranks = ranks.barrier, ranks.max

    pcpm.build()
    pcpm.lib()
    rp, col = make_graph(a)
    n, m = rp.size - 1, int(rp[-1])
    stream = torch.cuda.current_stream()

    d_rp, d_col = pcpm.to_device_csr(rp, col)
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    g = pcpm.PNG(d_rp, d_col, a.part_size, gather_windows=layout_option(a))
    build_ms = (time.perf_counter() - b0) * 1e3
    del d_rp, d_col
    info = g.info

    g.reset()
    g.iterate(a.d, a.warmup, sync=False, mode=a.mode)
    torch.cuda.synchronize()

    sampler = ClockSampler(local).start()
    time.sleep(0.2)
    barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    kms = g.iterate_timed(a.d, a.steps, mode=a.mode)  # per-kernel CUDA events on `stream`
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    barrier()
    clocks = sampler.stop(t0, t1)
    bracket_ms = ev0.elapsed_time(ev1)
    iter_ms = max_over_ranks(kms["span"] / a.steps)
    value = ranks.aggregate_gteps(m, iter_ms * 1e-3)

    # roofline of the kernel with the largest share of the time
    ab = algorithmic_bytes(info, a.mode)
    dom = max(PHASES, key=lambda p: kms[p])
    dom_ms = kms[dom] / a.steps
    peak, peak_src = measured_peaks()
    achieved = ab[dom] / (dom_ms * 1e-3) / 1e9
    wl = workload_name(a)
    kname = dom + (" (fused: gather, apply, next scatter)" if a.mode == "fused" and dom == "gather_apply" else "")
    traffic, traffic_note = recorded_traffic(dom, a.gather_layout, ab[dom])
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": traffic, "traffic_source": traffic_note, "algorithmic_bytes": ab[dom]}
    iter_bytes = sum(ab.values())

    # The other iteration form, timed the same way: two-phase gives the
    # paper's scatter / gather split (Table execTime analogue).
    other = None
    if not a.no_two_phase:
        om = "two_phase" if a.mode == "fused" else "fused"
        tp_steps = max(3, min(a.steps, 50))
        g.iterate(a.d, 3, sync=False, mode=om)
        tms = g.iterate_timed(a.d, tp_steps, mode=om)
        tab = algorithmic_bytes(info, om)
        other = {"mode": om, "iters": tp_steps, "ms_per_iter": tms["span"] / tp_steps,
                 "gteps": m / (tms["span"] / tp_steps * 1e-3) / 1e9}
        for ph in PHASES:
            ms = tms[ph] / tp_steps
            other[ph] = {"ms": ms, "gbs": tab[ph] / (ms * 1e-3) / 1e9 if ms > 0 else None,
                         "frac": tab[ph] / (ms * 1e-3) / 1e9 / peak if ms > 0 else None}

    out = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": iter_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl, "n": n, "m": m, "part_size": a.part_size, "k": info["num_partitions"],
                   "num_updates": info["num_updates"], "r": info["compression_ratio"], "d": a.d,
                   "gather_units": info["gather_units"], "gather_cluster": info["gather_cluster"],
                   "gather_runs": info["gather_runs"], "merged_adds": info["merged_adds"],
                   "gather_layout": a.gather_layout, "num_windows": info["num_windows"],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "no flush: each iteration moves ~%.2f GB, > 129 MB L2" % (iter_bytes / 1e9)},
        "roofline": roofline,
        "phase_ms_per_iter": {p: kms[p] / a.steps for p in PHASES},
        "hbm_gbs_achieved": iter_bytes / (iter_ms * 1e-3) / 1e9,
        "bytes_per_edge": {"algorithmic": iter_bytes / m, "eq5_model": eq5_bytes(info) / m},
        "mode": a.mode,
        "other_mode": other,
        "bracket_ms_per_step": bracket_ms / a.steps,
        "build_ms": build_ms,
        "clocks": clocks,
        "gpu_launches": 2 * a.steps,
    }

    if not a.no_converge:
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        _, its, res = g.pagerank(a.d, max_iters=300, tol=1e-7, mode=a.mode)
        torch.cuda.synchronize()
        out["time_to_residual"] = {"tol": 1e-7, "iters": its, "ms": (time.perf_counter() - c0) * 1e3,
                                   "final_residual": res, "reached": res < 1e-7, "start": "uniform"}
    g.close()

    if not a.no_e2e:
        e2e_iters = 20
        prp = torch.empty(n + 1, dtype=torch.int32, pin_memory=True)
        pcol = torch.empty(max(m, 1), dtype=torch.int32, pin_memory=True)
        pout = torch.empty(n, dtype=torch.float32, pin_memory=True)
        prp.numpy()[:] = rp.view(np.int32)
        pcol.numpy()[:m] = col.view(np.int32)
        hrp, hcol, hout = prp.numpy().view(np.uint32), pcol.numpy().view(np.uint32)[:m], pout.numpy()
        pcpm.pagerank_host(hrp, hcol, a.part_size, a.d, 3, pr_out=hout, mode=a.mode)  # warm-up call
        barrier()
        walls = []
        for _ in range(3):
            e0 = time.perf_counter()
            pcpm.pagerank_host(hrp, hcol, a.part_size, a.d, e2e_iters, pr_out=hout, mode=a.mode)
            walls.append(time.perf_counter() - e0)
        wall = max_over_ranks(statistics.median(walls))
        out["e2e"] = {"value": world * m * e2e_iters / wall / 1e9, "unit": "GTEPS",
                      "h2d_bytes_per_step": (n + 1 + m) * 4 / e2e_iters, "d2h_bytes_per_step": n * 4 / e2e_iters,
                      "call": "pcpm_pagerank_host: H2D CSR (pinned) + PNG build + %d %s iterations + D2H ranks"
                              % (e2e_iters, a.mode), "wall_ms_per_call": wall * 1e3}

    # Reduced-precision update bins (not in the paper): speed, bytes per edge,
    # and the first iteration's distance to the FP64 oracle's (below).
    first_iter, conv_ranks = {}, {}
    if not a.no_update_dtypes:
        d_rp, d_col = pcpm.to_device_csr(rp, col)
        dts = {}
        for dt_name in ("f32", "f16", "bf16"):
            gu = pcpm.PNG(d_rp, d_col, a.part_size, update_dtype=dt_name, gather_windows=layout_option(a))
            iu = gu.info
            gu.reset()
            gu.iterate(a.d, 1, mode=a.mode)
            first_iter[dt_name] = gu.ranks().cpu().numpy()
            gu.iterate(a.d, 3, sync=False, mode=a.mode)
            ksteps = max(3, min(a.steps, 100))
            tu = gu.iterate_timed(a.d, ksteps, mode=a.mode)
            abu = algorithmic_bytes(iu, a.mode)
            dts[dt_name] = {"gteps": m / (tu["span"] / ksteps * 1e-3) / 1e9, "ms_per_iter": tu["span"] / ksteps,
                            "phase_ms": {p: tu[p] / ksteps for p in PHASES},
                            "bytes_per_edge": sum(abu.values()) / m, "update_bytes": iu["update_bytes"]}
            if not a.no_converge:
                # time to the same L1 change as the FP32 solve, from the uniform start
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                xr, its, res = gu.pagerank(a.d, max_iters=300, tol=1e-7, mode=a.mode)
                e1.record()
                torch.cuda.synchronize()
                dts[dt_name]["time_to_residual"] = {"tol": 1e-7, "iters": its, "ms": e0.elapsed_time(e1),
                                                    "final_residual": res, "reached": res < 1e-7}
                conv_ranks[dt_name] = xr.cpu().numpy()
                if dt_name != "f32":  # delta iterations with rounding feedback (PCPM_DELTA)
                    torch.cuda.synchronize()
                    e0.record()
                    xd, itd, resd = gu.pagerank(a.d, max_iters=300, tol=1e-7, mode="delta")
                    e1.record()
                    torch.cuda.synchronize()
                    dts[dt_name]["time_to_residual_delta"] = {"tol": 1e-7, "iters": itd, "ms": e0.elapsed_time(e1),
                                                              "final_residual": resd, "reached": resd < 1e-7}
                    conv_ranks[dt_name + "_delta"] = xd.cpu().numpy()
            gu.close()
        del d_rp, d_col
        out["update_dtypes"] = dts

    if not a.no_spmv:
        out["spmv"] = spmv_leg(a, rp, col, m)

    if not a.no_warm_start:
        out["warm_start"] = warm_start_leg(a, rp, col)

    if not a.no_batched:
        out["batched"] = batched_leg(a)

    if not a.no_ppr:
        out["ppr"] = ppr_leg(a)

    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"], y_ref = cpu_oracle_baseline(rp, col, a.d)
        for dt_name, x1 in first_iter.items():
            out["update_dtypes"][dt_name]["l1_first_iteration_vs_fp64_oracle"] = float(
                np.abs(x1.astype(np.float64) - y_ref).sum())
        if "f32" in conv_ranks:  # converged ranks of each format against the FP32 solve's
            for key, xr in conv_ranks.items():
                dt_name, leg = (key[:-6], "time_to_residual_delta") if key.endswith("_delta") else (key, "time_to_residual")
                out["update_dtypes"][dt_name][leg]["l1_vs_f32_converged"] = float(
                    np.abs(xr.astype(np.float64) - conv_ranks["f32"].astype(np.float64)).sum())
    ranks.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def run_sharded(a):
    """N > 1 ranks: one graph split by destination partitions over the ranks
    (pcpm_build_shard), with NCCL exchanging the new ranks' slices and the two
    FP64 sums after every iteration. The whole graph's edges are processed per
    step whatever N is, so the scaling is strong."""
    import torch
    import torch.distributed as dist

    import paper_1709_07122_gb300 as pcpm
    from paper_1709_07122_gb300.sharded import ShardedPageRank

    rank, world, local = dist_env()
    if a.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    pcpm.build()
    pcpm.lib()
    rp, col = make_graph(a)  # the same seed on every rank: the same graph
    n, m = rp.size - 1, int(rp[-1])
    stream = torch.cuda.current_stream()

    def tmax(x):
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    d_rp, d_col = pcpm.to_device_csr(rp, col)
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    solver = ShardedPageRank(d_rp, d_col, a.part_size, gather_windows=layout_option(a))
    torch.cuda.synchronize()
    build_ms = tmax((time.perf_counter() - b0) * 1e3)
    del d_rp, d_col
    info = solver.png.info
    solver.reset()
    for _ in range(a.warmup):
        solver.step(a.d)
    torch.cuda.synchronize()

    sampler = ClockSampler(local).start()
    time.sleep(0.2)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(a.steps):
        solver.step(a.d)
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    dist.barrier()
    clocks = sampler.stop(t0, t1)
    iter_ms = tmax(ev0.elapsed_time(ev1) / a.steps)

    out = {
        "metric": METRIC, "value": m / (iter_ms * 1e-3) / 1e9, "unit": "GTEPS", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": iter_ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": n, "m": m, "part_size": a.part_size,
                   "k": info["num_partitions"], "d": a.d, "gather_layout": a.gather_layout,
                   "parallelism": f"destination shards x{world} (NCCL all-gather of ranks, FP64 all-reduce)",
                   "partition_cuts": [int(c) for c in solver.part_bounds],
                   "l2": "no flush: each iteration moves > 129 MB per GPU"},
        "build_ms": build_ms,
        "clocks": clocks,
        "gpu_launches": 3 * a.steps,
    }
    solver.close()

    if not a.no_e2e:
        e2e_iters = 20
        prp = torch.empty(n + 1, dtype=torch.int32, pin_memory=True)
        pcol = torch.empty(max(m, 1), dtype=torch.int32, pin_memory=True)
        pout = torch.empty(n, dtype=torch.float32, pin_memory=True)
        prp.numpy()[:] = rp.view(np.int32)
        pcol.numpy()[:m] = col.view(np.int32)
        walls = []
        for rep in range(3):
            dist.barrier()
            e0 = time.perf_counter()
            g_rp = prp.to("cuda", non_blocking=True)
            g_col = pcol.to("cuda", non_blocking=True)
            sv = ShardedPageRank(g_rp, g_col, a.part_size, gather_windows=layout_option(a))
            del g_rp, g_col
            x, _, _ = sv.pagerank(a.d, max_iters=e2e_iters)
            pout.copy_(x)
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - e0)
            sv.close()
        wall = tmax(statistics.median(walls))
        out["e2e"] = {"value": m * e2e_iters / wall / 1e9, "unit": "GTEPS",
                      "h2d_bytes_per_step": (n + 1 + m) * 4 / e2e_iters, "d2h_bytes_per_step": n * 4 / e2e_iters,
                      "call": "ShardedPageRank from pinned host CSR: H2D, shard build, %d iterations with "
                              "exchange, D2H ranks (every rank)" % e2e_iters, "wall_ms_per_call": wall * 1e3}
    dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)
    if dist_env()[1] > 1:
        return run_sharded(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
