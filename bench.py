"""Benchmark: graph Quantum Clustering on the DC-SBM N=16384 workload with the
16-value sigma sweep (one step = all-source BFS + histogram, potentials for 16
sigma values, descent and roots for each).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Other workloads, each printing its own JSON line: sbm262144 (one SBM of
262,144 nodes, sigma 1.5, the same line format; its CPU baseline is a bounded
sample scaled to the whole graph), directed16384 (a directed planted
partition, same format), batch4096 (4096 small graphs, batched plan vs the
plain path), serve (a Poisson request stream through the serving loop,
p50/p99), adjacency16384 (the distance-0/1/M mode), weighted16384 (weighted
shortest-path distances), fig3 (complete graphs of growing n, GPU vs oracle)
and quality (modularity, ARI, FMI, NMI over the sigma sweep on planted
partitions).

Prints one JSON line.  `value` is clusterings/s (one clustering = one label
vector for one (graph, sigma) pair) over all ranks, timed on the device with
CUDA events, inputs resident in HBM, L2 flushed (256 MiB write) before every
timed step.  On one GPU the default line also carries the rest of the headline
metric: `batch4096` (the batched plan against the plain one-graph-at-a-time
form, labels compared) and `serve` (p50/p99 latency of the Poisson request
stream, throughput against serial plain solves, labels compared, four
large-request workers at 40 % of the SMs each), with `serve_low_latency` the
same stream where two workers split 80 % of the SMs among the large requests
running; --no-extra leaves them out.  `e2e` is the same metric through the public API with host
buffers: one qc_cluster call per step takes the pinned host CSR to the device, validates it,
solves and writes the labels back to pinned host memory (`graph_object_ms_per_step`: the same
through qc_graph_create + qc_solve + a copy).
`--impl reference` times the CPU oracle (test infrastructure, plain C) on the
same workload instead.  With --gpus N > 1 each rank runs an independent replica
(the single-graph workload is not sharded) and rank 0 reports the total.
"""
from __future__ import annotations

import argparse
import ctypes
import faulthandler
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

WORKLOAD = ("dcsbm-16384: degree-corrected SBM, N=16384, 32 equal communities, power-law expected "
            "degrees (density exponent 2.5, mean 16, max 512), mixing 0.1, seed 1; sigma sweep of 16 "
            "values log-spaced 0.5-4.0 reusing one histogram")
METRIC = "clusterings/s"
PROFILE = os.path.join(ROOT, "profiles", "bfs_dcsbm16384.md")

# single-graph workloads: generator, description, the ncu summary holding the BFS
# kernel's DRAM traffic per launch, and how many nodes the CPU baseline samples
# (None: the whole workload)
SINGLE = {
    "dcsbm16384": {"make": lambda: gg.dcsbm16384(), "desc": WORKLOAD, "profile": PROFILE,
                   "cpu_sample_nodes": None, "steps": 200},
    "directed16384": {"make": lambda: (gg.directed_planted_partition(16384, 32, 16.0 * 0.9 / 511,
                                                                     16.0 * 0.1 / (16384 - 512), gg.rng(5, 1),
                                                                     name="dpp-16384"), gg.sigma_sweep16()),
                      "desc": ("directed16384: directed planted partition, N=16384, 32 blocks of 512, "
                               "mean out-degree 16, mixing 0.1, seed 5; the 16-value sigma sweep"),
                      "profile": None, "cpu_sample_nodes": None, "steps": 200},
    "sbm262144": {"make": lambda: gg.sbm262144(),
                  "desc": ("sbm-262144: SBM, N=262144, 256 equal communities of 1024, mean degree 20, "
                           "mixing 0.15, seed 2; sigma 1.5"),
                  "profile": os.path.join(ROOT, "profiles", "bfs_sbm262144.md"),
                  "cpu_sample_nodes": 512, "steps": 3},
}
KERNEL_SRC = [os.path.join(ROOT, "paper_2305_14641_gb300", "csrc", f) for f in ("bfs.cu", "qc_device.cuh")]


def kernel_source_sha256() -> str:
    """sha256 over the sources the BFS kernel is built from, in a fixed order."""
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        h.update(open(path, "rb").read())
    return h.hexdigest()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks of the process group (x itself when there is none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: float, steps: int, world: int, max_total_ms: float) -> float:
    """Units per second for the whole job: every rank runs `steps` steps of
    `units_per_step` (replicas), timed by the slowest rank."""
    return world * units_per_step * steps / (max_total_ms / 1000.0)


def gteps_edges(graph) -> float:
    """sum over sources of the undirected edges in the source's component (for a
    directed graph: the arcs of its weakly connected component, an upper bound)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    n = graph.n
    a = csr_matrix((np.ones(graph.nnz), graph.col_idx, graph.row_ptr), shape=(n, n))
    _, comp = connected_components(a, directed=False)
    size = np.bincount(comp)
    rows = np.repeat(np.arange(n), graph.degrees())
    edges = np.bincount(comp[rows], minlength=len(size)) / (1.0 if graph.directed else 2.0)
    return float((size * edges).sum())


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def profile_value(key: str, path=PROFILE):
    """A figure recorded in the committed ncu summary (`key: value`), if the summary
    was taken on the current kernel source (else None)."""
    if not path or not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    if kernel_source_sha256() != h.group(1):
        return None
    return float(m.group(1))


def profile_traffic(path=PROFILE):
    """dram bytes per launch from the committed ncu summary (None if stale)."""
    return profile_value("traffic_bytes_per_launch", path)


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def run_cpu_oracle(graph, sigmas, threads, sample_nodes=None):
    """Seconds the oracle takes for one solve of the workload.  With sample_nodes,
    the per-source BFS runs from that many evenly spaced nodes only and its time
    is scaled by n / sample_nodes; potentials, descent and roots then run on all
    n nodes over the sampled histogram rows repeated to n rows (the same
    per-node work)."""
    import oracle
    if sample_nodes is None or sample_nodes >= graph.n:
        t0 = time.perf_counter()
        oracle.solve(graph, sigmas, threads=threads)
        return time.perf_counter() - t0
    nodes = np.linspace(0, graph.n - 1, sample_nodes).astype(np.int32)
    t0 = time.perf_counter()
    h = oracle.histograms(graph, nodes, threads=threads)
    t_bfs = (time.perf_counter() - t0) * graph.n / sample_nodes
    full = np.ascontiguousarray(np.resize(h, (graph.n, h.shape[1])))
    t0 = time.perf_counter()
    for s in sigmas:
        V = oracle.potential(full, s)
        p, _ = oracle.ggd_parent(graph, V)
        oracle.find_centers(p)
    return t_bfs + time.perf_counter() - t0


def cpu_sample_text(graph, sigmas, sample_nodes):
    if sample_nodes is None or sample_nodes >= graph.n:
        return (f"one full solve of the workload: queue BFS from all {graph.n} sources, histograms, "
                f"{len(sigmas)} potential(s), descent, roots")
    return (f"queue BFS from {sample_nodes} evenly spaced sources of {graph.n}, time scaled by "
            f"{graph.n}/{sample_nodes}; then potential, descent and roots over all {graph.n} nodes")


def bench_reference(args, graph, sigmas, spec):
    """The oracle, as it stands, on the host cores: each step one solve of the workload
    (a bounded sample of it, scaled, where the whole would take minutes)."""
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return
    threads = oracle.default_threads()
    oracle.build()
    sample = spec["cpu_sample_nodes"]
    for _ in range(args.warmup):
        run_cpu_oracle(graph, sigmas, threads, sample)
    times = [run_cpu_oracle(graph, sigmas, threads, sample) for _ in range(args.steps)]
    total = sum(times)
    value = len(sigmas) * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
        "config": {"workload": spec["desc"], "n": graph.n, "nnz": graph.nnz, "sigmas": len(sigmas)},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                         "sample": cpu_sample_text(graph, sigmas, sample)},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_ours(args, graph, sigmas, spec):
    import torch
    import paper_2305_14641_gb300 as qc

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    # scratch from the stream-ordered CUDA pool: no Python callback per allocation
    ctx = qc.Context(local, allocator="cuda")
    S = len(sigmas)
    n = graph.n

    # device-resident inputs
    g = qc.Graph.from_graph(ctx, graph)
    V = torch.empty((S, n), dtype=torch.float64, device=dev)
    labels = torch.empty((S, n), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solve_step():
        g.drop_histogram()
        g.solve(sigmas, V_out=V, labels_out=labels, counts=False)

    plan = None
    if args.step == "plan":
        # the whole step (BFS from the resident CSR, 16 potentials, descent, roots)
        # captured once into CUDA graphs and replayed
        plan = qc.SweepPlan(g, sigmas, V=V, labels=labels)
        step = plan.run
    else:
        step = solve_step

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, each bracketed by events after an L2 flush
    launches0 = ctx.launch_count()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = ctx.launch_count() - launches0
    # the BFS kernel's own figures: the same steps through the single-graph path in
    # timing mode (CUDA events around each BFS launch, device timestamps per level)
    ctx.set_timing(True)
    ctx.kernel_stats("bfs_level", reset=True)
    for lvl in range(n + 2):
        if ctx.kernel_stats(f"bfs_pass_{lvl}", reset=True)["launches"] == 0 and lvl > 2:
            break
    for k in range(min(args.steps, 20)):
        flush.fill_(k & 0xff)
        solve_step()
    torch.cuda.synchronize()
    kstats = ctx.kernel_stats("bfs_level", reset=True)
    kstats_steps = min(args.steps, 20)
    # per-level device time inside the BFS launch (globaltimer stamps at each grid barrier);
    # level 1 is the set-up that writes the rows of levels 0-1
    level_us = {}
    for lvl in range(1, n + 2):
        st = ctx.kernel_stats(f"bfs_pass_{lvl}", reset=True)
        if st["launches"] == 0:
            break
        level_us[lvl] = round(1000.0 * st["total_ms"] / st["launches"], 2)
    ctx.set_timing(False)
    ctx_l2 = {"stream": ctx.l2_read_gbs(48 << 20), "random512": ctx.l2_read_gbs(48 << 20, random_segments=True)}
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(S, args.steps, world, total_ms)
    plan_info = plan.info() if plan is not None else None
    if plan is not None:
        plan.close()

    # end to end through the public API with host buffers
    rp_h = torch.from_numpy(graph.row_ptr).pin_memory()
    ci_h = torch.from_numpy(graph.col_idx).pin_memory()
    lab_h = torch.empty((S, n), dtype=torch.int32).pin_memory()
    h2d = rp_h.numel() * 4 + ci_h.numel() * 4
    d2h = lab_h.numel() * 4

    rp_np, ci_np = rp_h.numpy(), ci_h.numpy()

    def e2e_step():
        # one library call: upload, validation, BFS, potentials, descent, labels to pinned host
        qc.cluster(ctx, rp_np, ci_np, sigmas, labels_out=lab_h, counts=False, directed=graph.directed)

    def composed_step():
        # the same through the graph object: create, solve, copy the labels back
        gg_ = qc.Graph(ctx, rp_np, ci_np, validate=True, directed=graph.directed)
        _, lab_d, _ = gg_.solve(sigmas, labels_out=labels, counts=False)
        lab_h.copy_(lab_d, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        gg_.close()

    def time_steps(step):
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        times = []
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return max_over_ranks(float(sum(times)), dev)

    e2e_ms = time_steps(e2e_step)
    if not np.array_equal(lab_h.numpy(), labels.cpu().numpy()):
        raise RuntimeError("end-to-end labels differ from the device-resident solve's")
    composed_ms = time_steps(composed_step)
    e2e_value = whole_job_rate(S, args.steps, world, e2e_ms)

    if rank == 0:
        peak, peak_kind = measured_peak_gbs()
        avg_ms = kstats["total_ms"] / kstats["launches"] if kstats["launches"] else None
        min_per_launch = kstats["min_bytes"] / kstats["launches"] if kstats["launches"] else None
        achieved = (min_per_launch / (avg_ms / 1000.0) / 1e9) if avg_ms else None
        traffic = profile_traffic(spec["profile"])
        l2_read = profile_value("l2_read_bytes_per_launch", spec["profile"])
        # L2 read throughput measured live by the library's probe (48 MiB buffer, resident in L2)
        l2_peak = ctx_l2["stream"]
        l2_peak_random = ctx_l2["random512"]
        l2_achieved = (l2_read / (avg_ms / 1000.0) / 1e9) if (l2_read and avg_ms) else None
        edges = gteps_edges(graph)
        bfs_ms = kstats["total_ms"] / kstats_steps
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            threads = oracle.default_threads()
            t = run_cpu_oracle(graph, sigmas, threads, spec["cpu_sample_nodes"])
            cpu = {"value": S / t, "unit": METRIC, "cores": threads, "kind": "oracle",
                   "sample": cpu_sample_text(graph, sigmas, spec["cpu_sample_nodes"]),
                   "seconds": t}
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64 bitsets / f64", "data": "synthetic",
            "config": {"workload": spec["desc"], "n": n, "nnz": graph.nnz, "sigmas": S,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "256 MiB buffer written between timed steps",
                       "allocator": "stream-ordered CUDA pool (cudaMallocAsync)",
                       "step": ("sweep plan: BFS, potentials, descent and roots captured in CUDA graphs, "
                                "replayed from the resident CSR" if plan_info else
                                "single-graph path (qc_solve) after dropping the cached histogram"),
                       "captured": plan_info["captured"] if plan_info else None},
            "gteps": edges * world * args.steps / (total_ms / 1000.0) / 1e9,
            "bfs_gteps": (edges / (bfs_ms / 1000.0) / 1e9) if bfs_ms > 0 else None,
            "roofline": {"kernel": "bfs_two_hop + bfs_persistent (one BFS launch of a source chunk)",
                         "bound": "hbm", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic,
                         "bytes_per_launch": min_per_launch,
                         "bytes_model": "compulsory HBM bytes per launch (a lower bound): CSR, node order, row "
                                        "bounds, components and per-word masks read once, histogram rows written "
                                        "once, and per level the open (node, tile) rows read and written beyond "
                                        "what L2 holds (counted on the device; the two-hop set-up's level-2 rows "
                                        "written once); bitset buffers that fit in L2 add nothing",
                         "model_bytes_per_launch": (kstats["model_bytes"] / kstats["launches"]
                                                    if kstats["launches"] else None),
                         "model": "pull-all upper bound: per level 8*wn*(E+3N) bitset bytes + CSR + one "
                                  "histogram row",
                         "launches": kstats["launches"], "avg_launch_ms": avg_ms,
                         # where the kernel works: bytes it reads from L2 per launch (ncu, same capture as
                         # `traffic`) over its launch time, against an L2-resident copy measured live
                         "l2": {"achieved": l2_achieved, "peak": l2_peak, "unit": "GB/s",
                                "frac": (l2_achieved / l2_peak) if l2_achieved else None,
                                "peak_random512": l2_peak_random,
                                "frac_random512": (l2_achieved / l2_peak_random) if l2_achieved else None,
                                "read_bytes_per_launch": l2_read,
                                "ncu_l2_throughput_frac": profile_value("l2_throughput_frac", spec["profile"]),
                                "peak_kind": "measured live: a 48 MiB buffer read through L2 only, streamed "
                                             "(peak) and as random 512-byte segments one per warp "
                                             "(peak_random512, the gather pattern)"}},
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps,
                    "call": "qc_cluster (host CSR in, host labels out, one call)",
                    "graph_object_ms_per_step": composed_ms / args.steps},
            "bfs_level_us": level_us,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
        }
    g.close()
    ctx.close()
    if rank == 0:
        if world == 1 and not args.no_extra:
            # the rest of the headline metric: batched vs plain, and the served form's latency
            line["batch4096"] = batch_summary(args)
            line["serve"] = serve_summary(args)
            # the same stream at the latency-oriented operating point: two large-request
            # workers whose requests split 80 % of the SMs among those running at once
            low = argparse.Namespace(**vars(args))
            low.large_workers, low.large_sm_share, low.divide_share = 2, 0.8, 1
            line["serve_low_latency"] = serve_summary(low)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


BATCH_WORKLOAD = ("batch4096: 4096 planted-partition graphs, N log-uniform in [32, 2048], 2-16 blocks, "
                  "p_in U(0.1, 0.5), p_out 0.02, sigma U(0.5, 3.0), seed 3; one persistent launch under a "
                  "captured CUDA graph")
SERVE_WORKLOAD = ("serve: Poisson arrivals at 200 requests/s of SBM graphs, N log-uniform in [64, 65536], "
                  "mean degree 12, 4-64 blocks, mixing 0.1, sigma U(0.5, 3.0), seed 4, 100 GB admission budget")


def batch_summary(args) -> dict:
    """Batched plan vs the plain form (one graph at a time through qc_solve), with
    the labels of every plain-solved graph compared with the batched ones."""
    import torch
    import paper_2305_14641_gb300 as qc
    graphs, sigmas = gg.planted_batch(args.batch_graphs)
    ctx = qc.Context(0)
    Gs = [qc.Graph.from_graph(ctx, g, validate=False) for g in graphs]
    t0 = time.perf_counter()
    plan = qc.BatchPlan(ctx, Gs, sigmas)
    plan_s = time.perf_counter() - t0
    for _ in range(max(args.warmup, 3)):
        plan.run(counts=False)
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    times = []
    launches0 = ctx.launch_count()
    steps = max(3, min(args.steps, 20))
    with ClockSampler(0) as clocks:
        for k in range(steps):
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run(counts=False)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    launches = (ctx.launch_count() - launches0) // steps
    batched = len(graphs) * steps / (sum(times) / 1000.0)
    batched_labels = plan.labels.cpu().numpy()
    # plain form: every graph through the single-graph path, one after another
    m = min(len(graphs), args.plain_graphs)
    for G, s in zip(Gs[:8], sigmas[:8]):
        G.solve([s], counts=False)
    torch.cuda.synchronize()
    plain_labels = []
    t0 = time.perf_counter()
    for G, s in zip(Gs[:m], sigmas[:m]):
        G.drop_histogram()
        plain_labels.append(G.solve([s], counts=False)[1])
    torch.cuda.synchronize()
    plain = m / (time.perf_counter() - t0)
    same = all(np.array_equal(lab.cpu().numpy()[0], batched_labels[plan.offsets[k]:plan.offsets[k] + graphs[k].n])
               for k, lab in enumerate(plain_labels))
    out = {"metric": "clusterings/s", "workload": BATCH_WORKLOAD, "graphs": len(graphs),
           "nodes": int(sum(g.n for g in graphs)), "directed_edges": int(sum(g.nnz for g in graphs)),
           "batched": batched, "ms_per_batch": sum(times) / len(times), "plain": plain,
           "batched_over_plain": batched / plain, "labels_identical_on_plain_sample": bool(same),
           "kernel_config": plan.config(), "gpu_launches_per_batch": launches,
           "plain_sample_graphs": m, "plan_seconds": plan_s, "steps": steps, "clocks": clocks.summary()}
    plan.close()
    for G in Gs:
        G.close()
    ctx.close()
    return out


def bench_batch(args):
    print(json.dumps(batch_summary(args)), flush=True)


def serve_summary(args) -> dict:
    """Open-loop Poisson stream through the server (p50/p99 latency over the
    requests after the warm-up ones), closed-loop throughput, and the same requests
    solved serially with the plain form (FIFO), whose labels must equal the served
    ones.  The serial run also records its BFS device time, which bounds what any
    form can reach while the large requests' BFS launches fill the GPU."""
    import threading as th
    import torch
    import paper_2305_14641_gb300 as qc
    reqs = gg.sbm_request_stream(args.requests)
    t_gen = time.perf_counter()
    graphs = [r.graph() for r in reqs]
    t_gen = time.perf_counter() - t_gen
    lat, results, served_labels = {}, {}, {}
    with qc.Server(0, large_workers=args.large_workers, large_sm_share=args.large_sm_share,
                   divide_share=args.divide_share) as srv:
        # warm up: a few requests of each kind
        for g, r in list(zip(graphs, reqs))[:8]:
            srv.wait(srv.submit(g.row_ptr, g.col_idx, r.sigma))
        ids = []

        def collector():
            for i in range(len(reqs)):
                while len(ids) <= i:
                    time.sleep(0.0005)
                res = srv.wait(ids[i])
                lat[i] = res["latency_ms"]
                results[i] = (res["n_clusters"], res["admit_ms"], res["batch_size"], res["start_ms"])
                served_labels[i] = res["labels"]

        col = th.Thread(target=collector)
        col.start()
        with ClockSampler(0) as clocks:
            # the arrival clock starts once the sampler is up, so no arrivals bunch up behind it
            t_start = time.perf_counter()
            for i, (g, r) in enumerate(zip(graphs, reqs)):
                delay = r.arrival_s - (time.perf_counter() - t_start)
                if delay > 0:
                    time.sleep(delay)
                ids.append(srv.submit(g.row_ptr, g.col_idx, r.sigma))
            col.join()
        open_wall = time.perf_counter() - t_start
        st_open = srv.stats()
        # closed loop: everything submitted at once
        t0 = time.perf_counter()
        cids = [srv.submit(g.row_ptr, g.col_idx, r.sigma) for g, r in zip(graphs, reqs)]
        for i in cids:
            srv.wait(i)
        closed = len(reqs) / (time.perf_counter() - t0)
    # serial plain solves of the same requests (FIFO), device-resident after upload
    ctx = qc.Context(0)
    for g, r in list(zip(graphs, reqs))[:8]:
        G = qc.Graph.from_graph(ctx, g)
        G.solve([r.sigma], counts=True)
        G.close()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.kernel_stats("bfs_level", reset=True)
    same = True
    t0 = time.perf_counter()
    service = []
    for i, (g, r) in enumerate(zip(graphs, reqs)):
        s0 = time.perf_counter()
        G = qc.Graph.from_graph(ctx, g)
        _, lab, _ = G.solve([r.sigma], counts=True)
        G.close()
        service.append(time.perf_counter() - s0)
        same = same and np.array_equal(lab.cpu().numpy()[0], served_labels[i])
    serial_wall = time.perf_counter() - t0
    serial = len(reqs) / serial_wall
    bfs = ctx.kernel_stats("bfs_level", reset=True)
    ctx.set_timing(False)
    ctx.close()
    # latency of the serial plain form under the same arrivals (FIFO queue simulation)
    free_at, serial_lat = 0.0, []
    for r, sv in zip(reqs, service):
        start = max(r.arrival_s, free_at)
        free_at = start + sv
        serial_lat.append(1000.0 * (free_at - r.arrival_s))
    warm = min(args.serve_warmup, len(reqs) - 1)
    keep = list(range(warm, len(reqs)))
    L = np.array([lat[i] for i in range(len(reqs))])
    big = [i for i in keep if results[i][2] == 0]
    small = [i for i in keep if results[i][2] > 0]

    def split(idx):
        if not idx:
            return None
        wait = np.array([results[i][3] for i in idx])
        run = np.array([lat[i] - results[i][3] for i in idx])
        return {"count": len(idx), "p50_ms": float(np.percentile(L[idx], 50)),
                "p99_ms": float(np.percentile(L[idx], 99)), "mean_wait_ms": float(wait.mean()),
                "mean_run_ms": float(run.mean()),
                "mean_serial_service_ms": float(1000 * np.mean([service[i] for i in idx]))}
    bfs_s = bfs["total_ms"] / 1000.0
    return {"metric": "clusterings/s", "workload": SERVE_WORKLOAD, "requests": len(reqs),
            "warmup_requests": warm, "large_workers": args.large_workers,
            "large_sm_share": args.large_sm_share, "divide_share": bool(args.divide_share),
            "served_open_loop_per_s": len(reqs) / open_wall,
            "p50_ms": float(np.percentile(L[keep], 50)), "p99_ms": float(np.percentile(L[keep], 99)),
            "served_closed_loop_per_s": closed, "serial_plain_per_s": serial,
            "served_over_serial_plain": closed / serial,
            "serial_plain_p50_ms": float(np.percentile(np.array(serial_lat)[keep], 50)),
            "serial_plain_p99_ms": float(np.percentile(np.array(serial_lat)[keep], 99)),
            "labels_identical_served_vs_plain": bool(same),
            # the serial run's BFS launches alone (CUDA events); every request's BFS still has
            # to run in any form, so requests / this time caps the served rate unless BFS
            # launches of different requests overlap on the GPU
            "serial_plain_bfs_device_s": bfs_s, "serial_plain_wall_s": serial_wall,
            "serial_plain_bfs_share": bfs_s / serial_wall if serial_wall > 0 else None,
            "ceiling_over_serial_if_bfs_serialised": (serial_wall / bfs_s) if bfs_s > 0 else None,
            "batched_requests": split(small), "worker_requests": split(big),
            "server_stats": {k: int(v) for k, v in st_open.items()}, "clocks": clocks.summary(),
            "generate_seconds": t_gen,
            "slowest": [{"n": reqs[i].n, "latency_ms": round(float(L[i]), 3),
                         "admit_ms": round(results[i][1], 3), "start_ms": round(results[i][3], 3),
                         "batch_size": results[i][2],
                         "serial_service_ms": round(1000 * service[i], 3)}
                        for i in sorted(keep, key=lambda i: -L[i])[:8]]}


def bench_serve(args):
    print(json.dumps(serve_summary(args)), flush=True)


def _device_steps(step, steps, flush, stream):
    """Mean CUDA-event milliseconds of `step` over `steps` runs, L2 flushed before each."""
    import torch
    times = []
    for k in range(steps):
        flush.fill_(k & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.mean(times))


def bench_adjacency(args):
    """The adjacency-distance mode (d = 0, 1 or M) on the dcsbm-16384 graph: 16 potentials,
    descent and roots per step; no BFS.  Also the potential kernel alone against HBM."""
    import torch
    import paper_2305_14641_gb300 as qc
    graph, sigmas = gg.dcsbm16384()
    ctx = qc.Context(0)
    g = qc.Graph.from_graph(ctx, graph)
    S, n = len(sigmas), graph.n
    V = torch.empty((S, n), dtype=torch.float64, device="cuda")
    lab = torch.empty((S, n), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        g.potential_adjacency(sigmas, 2.0, out=V)
        g.ggd_labels(V, out=lab, counts=False)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    with ClockSampler(0) as clocks:
        ms = _device_steps(step, args.steps, flush, stream)
    launches = ctx.launch_count() - launches0
    pot_ms = _device_steps(lambda: g.potential_adjacency(sigmas, 2.0, out=V), args.steps, flush, stream)
    peak, peak_kind = measured_peak_gbs()
    pot_bytes = 4.0 * (n + 1) + 8.0 * n * S
    line = {"metric": METRIC, "workload": "adjacency16384: " + WORKLOAD + "; distance 0 / 1 / M = 2",
            "value": S / (ms / 1000.0), "unit": METRIC, "ms_per_step": ms, "steps": args.steps,
            "gpu_launches": launches, "clocks": clocks.summary(),
            "potential_kernel": {"ms": pot_ms, "bytes": pot_bytes,
                                 "achieved_gbs": pot_bytes / (pot_ms / 1000.0) / 1e9, "peak": peak,
                                 "peak_kind": peak_kind,
                                 "note": "launch-bound: 2.2 MB per launch; the event span includes launch latency"}}
    print(json.dumps(line), flush=True)
    g.close()
    ctx.close()


def bench_weighted(args):
    """Weighted shortest-path distances on the dcsbm-16384 graph with weights drawn
    U(0.5, 2.0): all-source shortest paths, 16 potentials, descent and roots per
    step; the oracle (Dijkstra per source) on a sample of sources, scaled."""
    import torch
    import oracle
    import paper_2305_14641_gb300 as qc
    graph, sigmas = gg.dcsbm16384()
    w = gg.edge_weights(graph, 0.5, 2.0, gg.rng(7, 1))
    ctx = qc.Context(0)
    g = qc.Graph.from_graph(ctx, graph)
    g.set_weights(w)
    S, n = len(sigmas), graph.n
    V = torch.empty((S, n), dtype=torch.float64, device="cuda")
    lab = torch.empty((S, n), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        g.potential_weighted(sigmas, out=V)
        g.ggd_labels(V, out=lab, counts=False)

    step()
    torch.cuda.synchronize()
    steps = max(2, min(args.steps, 10))
    launches0 = ctx.launch_count()
    with ClockSampler(0) as clocks:
        ms = _device_steps(step, steps, flush, stream)
    launches = (ctx.launch_count() - launches0) // steps
    # the shortest paths with a single sigma, to split the step between paths and sums
    one_ms = _device_steps(lambda: g.potential_weighted(sigmas[:1], out=V[:1]), steps, flush, stream)
    cpu = None
    if not args.no_cpu_baseline:
        oracle.build()
        threads = oracle.default_threads()
        t0 = time.perf_counter()
        oracle.potential_weighted(graph, w, sigmas, threads=threads)
        cpu_s = time.perf_counter() - t0
        cpu = {"value": S / cpu_s, "unit": METRIC, "cores": threads, "kind": "oracle", "seconds": cpu_s,
               "sample": f"the whole potential: Dijkstra from all {n} sources and the pair sums for "
                         f"{S} sigma values (descent not included)"}
    line = {"metric": METRIC, "workload": "weighted16384: the dcsbm-16384 graph with edge weights "
                                          "U(0.5, 2.0), seed 7; 16 sigma values",
            "value": S / (ms / 1000.0), "unit": METRIC, "ms_per_step": ms, "steps": steps,
            "ms_paths_and_one_sigma": one_ms,
            "gpu_launches_per_step": launches, "clocks": clocks.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    g.close()
    ctx.close()


def bench_fig3(args):
    """Fully-connected graphs of growing n (the workload of the paper's GPU-vs-CPU figure):
    time per clustering (sigma = 1) on the GPU, hop and adjacency distance, and the oracle
    on the host cores (adjacency mode whole; hop mode from 32 sampled sources, scaled)."""
    import torch
    import oracle
    import paper_2305_14641_gb300 as qc
    oracle.build()
    threads = oracle.default_threads()
    ctx = qc.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    for n in (512, 1024, 2048, 4096, 8192):
        graph = gg.complete(n)
        g = qc.Graph.from_graph(ctx, graph, validate=False)
        V = torch.empty((1, n), dtype=torch.float64, device="cuda")
        lab = torch.empty((1, n), dtype=torch.int32, device="cuda")

        def hop():
            g.drop_histogram()
            g.solve([1.0], V_out=V, labels_out=lab, counts=False)

        def adj():
            g.potential_adjacency([1.0], 2.0, out=V)
            g.ggd_labels(V, out=lab, counts=False)

        for f in (hop, adj):
            for _ in range(3):
                f()
        torch.cuda.synchronize()
        steps = max(3, min(args.steps, 20))
        hop_ms = _device_steps(hop, steps, flush, stream)
        adj_ms = _device_steps(adj, steps, flush, stream)
        t0 = time.perf_counter()
        Va = oracle.potential_adjacency(graph, 1.0, 2.0)
        oracle.find_centers(oracle.ggd_parent(graph, Va)[0])
        cpu_adj = 1000.0 * (time.perf_counter() - t0)
        cpu_hop = 1000.0 * run_cpu_oracle(graph, [1.0], threads, 32)
        rows.append({"n": n, "directed_edges": graph.nnz, "gpu_hop_ms": hop_ms, "gpu_adjacency_ms": adj_ms,
                     "cpu_hop_ms": cpu_hop, "cpu_adjacency_ms": cpu_adj})
        g.close()
    print(json.dumps({"workload": "fig3: complete graphs K_n, sigma 1, one clustering per step", "cpu_cores": threads,
                      "rows": rows}), flush=True)
    ctx.close()


# (nodes, undirected edges, classes) the paper reports for its datasets; the graphs
# below are planted partitions of those shapes, not the datasets
QUALITY_SHAPES = {"cora-shaped": (2708, 5278, 7), "citeseer-shaped": (3327, 4676, 6),
                  "wiki-shaped": (2405, 12761, 17), "cora-ml-shaped": (2995, 8158, 7),
                  "karate-shaped": (34, 78, 2)}


def bench_quality(args):
    """Quality against the planted communities over the 16-value sigma sweep (the
    analogue of the paper's sigma-sensitivity figure on synthetic stand-ins):
    modularity, ARI, FMI, NMI (computed on the device) and the number of clusters
    per sigma; solve_ms covers the solve and the 16 measurements."""
    import torch
    import paper_2305_14641_gb300 as qc
    sigmas = gg.sigma_sweep16()
    ctx = qc.Context(0)
    out = {}
    for name, (n, m, k) in QUALITY_SHAPES.items():
        graph = gg.sbm_mean_degree(n, k, 2.0 * m / n, 0.2, gg.rng(6, n), name=name)
        g = qc.Graph.from_graph(ctx, graph)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, labels, counts = g.solve(sigmas)
        truth = torch.as_tensor(graph.block, device="cuda")
        curve = []
        for s, lab, c in zip(sigmas, labels, counts):
            m = qc.quality(ctx, lab, graph=g, truth=truth, n_truth=int(graph.block.max()) + 1)
            curve.append({"sigma": round(s, 4), "clusters": int(c), "modularity": m["modularity"],
                          "ari": m["ari"], "fmi": m["fmi"], "nmi": m["nmi"]})
        secs = time.perf_counter() - t0
        best = max(curve, key=lambda r: r["nmi"])
        out[name] = {"n": n, "edges": graph.nnz // 2, "planted": k, "solve_ms": 1000.0 * secs,
                     "best_by_nmi": best, "curve": curve}
        g.close()
    print(json.dumps({"workload": "quality: planted partitions (mixing 0.2) of the paper's dataset shapes; "
                                  "16 sigma values 0.5-4.0", "graphs": out}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200; 3 for sbm262144)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--step", choices=["plan", "solve"], default="plan",
                    help="default workload: replay the captured sweep plan, or the single-graph path")
    ap.add_argument("--workload", choices=["dcsbm16384", "sbm262144", "directed16384", "batch4096", "serve",
                                           "adjacency16384", "weighted16384", "fig3", "quality"],
                    default="dcsbm16384")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--plain-graphs", type=int, default=512)
    ap.add_argument("--requests", type=int, default=4000)
    ap.add_argument("--serve-warmup", type=int, default=200,
                    help="requests at the start of the stream left out of the latency figures")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: leave out the batch4096 and serve sub-lines")
    ap.add_argument("--large-workers", type=int, default=4)
    ap.add_argument("--large-sm-share", type=float, default=0.4)
    ap.add_argument("--divide-share", type=int, default=0,
                    help="serve: split the large-request SM share among the large requests running")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = SINGLE[args.workload]["steps"] if args.workload in SINGLE else 200
    if args.workload == "batch4096":
        return bench_batch(args)
    if args.workload == "serve":
        return bench_serve(args)
    if args.workload == "adjacency16384":
        return bench_adjacency(args)
    if args.workload == "fig3":
        return bench_fig3(args)
    if args.workload == "weighted16384":
        return bench_weighted(args)
    if args.workload == "quality":
        return bench_quality(args)
    spec = SINGLE[args.workload]
    graph, sigmas = spec["make"]()
    if args.impl == "reference":
        bench_reference(args, graph, sigmas, spec)
    else:
        bench_ours(args, graph, sigmas, spec)


if __name__ == "__main__":
    # a crash in native code prints the Python stack of every thread to stderr
    faulthandler.enable()
    main()
