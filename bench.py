#!/usr/bin/env python
"""Benchmark: HyperBall GEdge-unions/s at p = 10 on the 236k-cell city graph.

One step is one whole analysis (Algorithm 1): counter initialisation, c_0,
d = 3 union passes (Eq. hll-union over the device-resident LEB128 CSR) with the
HLL estimate and Eq. sumD after each, and Visual Mean Depth.  The metric is
GEdge-unions/s = (passes x directed edges) / seconds / 1e9, the unit the
paper's BFS-phase times translate to (Sec. 4.3 breakdown table).

Workload (synthetic stand-in for the paper's 235,983-cell Valdivia graph,
which is not available): the seeded 520 x 520 urban-block grid of
workloads.city(2), 236,693 main-component cells, ~4.63e9 directed edges,
~4.7 GB of compressed CSR, built on the GPU before timing.

Arms:
  default           the CUDA library; `value` is device-timed with the CSR and
                    workspace resident, `e2e` goes through the public C API
                    with host buffers (CSR copied in and results copied out
                    every step).
  --impl reference  the CPU oracle as it stands, on the host cores, over a
                    bounded sample of the same workload (one union pass over
                    sampled nodes per step).

Extras of the default run (N = 1, after the timed region): e2e, unlimited
depth, sweeps, the oracle's union-pass throughput on the city sample and its
whole analysis on the medium graph beside the GPU's, and compact records of
the batched workload (256 graphs, against one-at-a-time runs) and the served
workload (2,000 Poisson requests per offered load at 0.5x, 0.9x and 1.5x,
against the measured one-at-a-time loop); --no-extras and --no-serve skip
them.  --mode batch and --mode serve print those records as their own lines.

Multi-GPU: the analysis does not shard without a cross-device exchange, so
`--gpus N` runs N independent replicas (weak scaling); value = all ranks'
edge unions / the slowest rank's time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "GEdge-unions/s at p=10 (236k-cell city graph, d=3)"
UNIT = "GEdge-unions/s"
CONFIGS = {
    "city": dict(grid=lambda: workloads.city(2), name="city 520x520 urban blocks, seed 2 (~236.7k cells, ~4.63e9 edges)"),
    "medium": dict(grid=lambda: workloads.medium(3), name="medium 220x220, seed 3 (~42.7k cells, ~4.2e8 edges)"),
    "tiny": dict(grid=lambda: workloads.tiny(1), name="tiny 32x32, seed 1 (903 cells)"),
}
PAPER_CONTEXT = {"paper_bfs_seconds_p10_d3_235983_cells_4.8e9_edges": 51.6,
                 "paper_derived_geu_per_s": 0.28,
                 "paper_hardware": "RTX 3080 Ti Laptop (sm_86), PCIe-streamed graph"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="city")
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU-baseline sample duration")
    ap.add_argument("--cpu-sample", type=int, default=256, help="sampled nodes for the CPU oracle")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, d=unlimited and CPU baseline")
    ap.add_argument("--slice-bytes", type=int, default=0, help="force the union slice width (0 = automatic)")
    ap.add_argument("--warps", type=int, default=0, help="force union warps per CTA (0 = automatic)")
    ap.add_argument("--order", choices=["raster", "hilbert"], default="raster", help="node numbering of the graph")
    ap.add_argument("--register-bits", type=int, default=8, choices=[8, 4],
                    help="8: uint8 registers; 4: the paper's packed 4-bit registers")
    ap.add_argument("--union-mode", type=int, default=0,
                    help="0 automatic, 1 one gather per neighbour, 2 per run of consecutive ids")
    ap.add_argument("--mode", choices=["metric", "batch", "serve"], default="metric",
                    help="metric: the headline analysis; batch: 256-graph batched workload; serve: Poisson requests")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests per offered load")
    ap.add_argument("--no-serve", action="store_true", help="skip the batch and serve legs of the default run")
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--lane-priority", type=int, default=0,
                    help="server: 1 favours the solo lane, -1 the batched")
    ap.add_argument("--solo-nodes", type=int, default=0, help="server: solo-lane threshold (0 = library default)")
    ap.add_argument("--batched-share", type=int, default=0,
                    help="server: percent of the batched lane's CTAs kept while a solo analysis runs (0 = all)")
    ap.add_argument("--backend", default="nccl")
    ap.add_argument("--autotune", action="store_true",
                    help="run the per-degree-bucket autotuner on the workload's graphs before timing")
    ap.add_argument("--hub-lookups", type=int, default=0, help="force the run-aware hub threshold (0 = automatic)")
    ap.add_argument("--l2-window", type=int, default=0, choices=[0, 1],
                    help="1: mark the union's table region persisting in L2 (access-policy window)")
    ap.add_argument("--first-pass", type=int, default=0, choices=[0, 1, 2],
                    help="pass 1: 0 automatic (scatter), 1 the union's gather, 2 the scatter")
    ap.add_argument("--track-changes", type=int, default=0, choices=[0, 1, 2],
                    help="change tracking: 0 automatic, 1 off, 2 every pass from the second")
    ap.add_argument("--group-nodes", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="grouped union: nodes per group (0 automatic = 4, 1 one node per warp)")
    ap.add_argument("--table-levels", type=int, default=0, choices=[0, 3, 5],
                    help="run-aware table rows per node: 5 (windows 1..16), 3 (1, 4, 16), 0 = automatic")
    ap.add_argument("--sharded", action="store_true",
                    help="N > 1: split one analysis over the ranks by register slice (strong scaling) instead of "
                         "running one replica per rank")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ----------------------------------------------------------------------------

class Dist:
    def __init__(self, backend):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def combine(units_local: float, seconds_local: float, dist: Dist):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    units = dist.sum(units_local)
    seconds = dist.max(seconds_local)
    return units, seconds


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------

class OracleSample:
    """One union pass of the CPU oracle over sampled nodes of the workload.

    The sampled nodes' neighbour lists come from the oracle's own visibility
    builder on the obstacle grid and its own encoder; the counters are its own
    initialisation.  Nothing here comes from the CUDA library."""

    def __init__(self, obst, p, seed, n_sample, rng_seed=12345):
        import oracle
        self.oracle = oracle
        self.p = p
        self.cores = oracle.default_threads()
        _, cells = oracle.main_component(obst)
        self.n = len(cells)
        rng = np.random.default_rng(rng_seed)
        self.sample = np.sort(rng.choice(self.n, min(n_sample, self.n), replace=False)).astype(np.int64)
        t0 = time.perf_counter()
        row_ptr_s, col = oracle.visibility_csr(obst, cells, nodes=self.sample, nthreads=self.cores)
        self.build_seconds = time.perf_counter() - t0  # the oracle's builder on the sampled sources
        counts = np.zeros(self.n, np.int64)
        counts[self.sample] = np.diff(row_ptr_s.astype(np.int64))
        row_ptr = np.zeros(self.n + 1, np.uint64)
        row_ptr[1:] = np.cumsum(counts)
        self.offsets, self.bytes = oracle.csr_encode(row_ptr, col)
        self.regs = oracle.hll_init(self.n, p, seed)
        self.edges = int(row_ptr[-1])

    def one_pass(self) -> tuple[float, int]:
        t0 = time.perf_counter()
        _, _, edges = self.oracle.union_pass(self.offsets, self.bytes, self.regs, self.p, nodes=self.sample,
                                             nthreads=self.cores)
        return time.perf_counter() - t0, edges

    def describe(self, reps) -> str:
        return (f"one Eq. hll-union pass (p={self.p}) over {len(self.sample)} sampled nodes of the "
                f"{self.n}-node graph ({self.edges} edge unions), repeated {reps}x; lists from the oracle's own "
                f"visibility builder")


def cpu_baseline(obst, args) -> dict:
    """Union-pass throughput of the oracle: one Eq. hll-union pass over sampled
    nodes of the workload, scaled to GEdge-unions/s (the whole analysis is timed
    on the medium graph by full_analysis_medium)."""
    s = OracleSample(obst, args.p, args.seed, args.cpu_sample)
    s.one_pass()  # warm caches
    total_t, total_e, reps = 0.0, 0, 0
    while total_t < args.cpu_seconds or reps < 1:
        t, e = s.one_pass()
        total_t += t
        total_e += e
        reps += 1
    return {"value": total_e / total_t / 1e9, "unit": UNIT, "cores": s.cores, "kind": "oracle",
            "sample": s.describe(reps), "seconds": total_t,
            "builder": {"sources": len(s.sample), "seconds": s.build_seconds,
                        "pair_tests_per_s": len(s.sample) * (s.n - 1) / s.build_seconds,
                        "what": "the oracle's visibility builder (supercover DDA per pair) for the sampled sources"}}


def full_analysis_medium(vga, torch, stream, p: int = 10, d: int = 3) -> dict:
    """Algorithm 1 in full (initialisation, c_0, d union passes with the
    estimator and Eq. sumD after each, mean depth) on the 42.7k-cell medium
    graph: the CPU oracle as it stands on all host cores, and the CUDA library
    on the same grid, with the mean depths compared node by node.  The oracle
    builds its own CSR from the obstacle grid; the library builds its own."""
    import oracle
    obst = CONFIGS["medium"]["grid"]()
    cores = oracle.default_threads()
    t0 = time.perf_counter()
    off, b, cells = oracle.build_graph(obst, nthreads=cores)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ref = oracle.hyperball(off, b, p, d, seed=0, nthreads=cores)
    cpu_s = time.perf_counter() - t0
    E = int(np.count_nonzero(np.asarray(b) < 0x80))  # one final (high-bit-clear) byte per LEB128 varint
    g = vga.vga_visibility_build(obst)
    md = torch.empty(max(g.n_nodes, 1), dtype=torch.float64, device="cuda")
    vga.hyperball_run_dev(g, p, d, 0, md, None, stream=stream)  # warm-up (lookup list)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    passes = vga.hyperball_run_dev(g, p, d, 0, md, None, stream=stream)
    f1.record(stream)
    torch.cuda.synchronize()
    gpu_s = f0.elapsed_time(f1) / 1e3
    same = bool(np.array_equal(md[: g.n_nodes].cpu().numpy(), ref["mean_depth"], equal_nan=True))
    g.free()
    return {"workload": CONFIGS["medium"]["name"], "p": p, "d": d, "N": len(cells), "E": E,
            "passes": ref["iterations"], "cores": cores,
            "cpu_seconds": cpu_s, "cpu_geu_per_s": ref["iterations"] * E / cpu_s / 1e9,
            "cpu_graph_build_seconds": build_s,
            "gpu_seconds": gpu_s, "gpu_geu_per_s": passes * E / gpu_s / 1e9, "gpu_passes": passes,
            "gpu_over_cpu": cpu_s / gpu_s, "mean_depth_bit_identical": same,
            "what": "the oracle's whole analysis (Alg. 1) on all host cores vs hyperball_run_dev on the GPU "
                    "(CUDA events), same grid, each side building its own CSR"}


def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return
    obst = CONFIGS[args.config]["grid"]()
    s = OracleSample(obst, args.p, args.seed, args.cpu_sample)
    for _ in range(args.warmup):
        s.one_pass()
    total_t, total_e = 0.0, 0
    for _ in range(args.steps):
        t, e = s.one_pass()
        total_t += t
        total_e += e
    value = total_e / total_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": CONFIGS[args.config]["name"], "p": args.p, "d": args.d, "seed": args.seed,
                       "N": s.n, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": s.cores, "kind": "oracle",
                             "sample": s.describe(args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def kernel_source_sha() -> str:
    """Hash of the union kernels' source: their device code (hb_device.cuh), the
    lookup and work-item declarations in vga_common.cuh, their definitions in
    hyperball.cu (host code there does not count), and the group-list builder
    in runs.cu (which decides what a grouped launch gathers)."""
    h = hashlib.sha256()

    def region(rel, start, end):
        with open(os.path.join(ROOT, rel), "rb") as f:
            src = f.read()
        a = src.find(start) if start else 0
        b = src.find(end, a) if end else len(src)
        h.update(src[a:b] if 0 <= a < b else src)

    region("paper_2604_08374_gb300/csrc/hb_device.cuh", None, None)
    region("paper_2604_08374_gb300/csrc/vga_common.cuh", b"constexpr int kRunLevels", b"// Work list of the run-aware")
    region("paper_2604_08374_gb300/csrc/hyperball.cu", b"// Eq. hll-union for one register slice, one warp per node",
           b"// Microbenchmark twin of hb_union_kernel")
    # how the grouped union's groups and their row lists are formed
    region("paper_2604_08374_gb300/csrc/runs.cu", b"// Merge key of a range lookup", None)
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, config: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; otherwise None."""
    path = os.path.join(ROOT, "profiles", "union_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None, None
    entry = rec.get(config, {})
    if entry.get("kernel") != kernel or entry.get("src_sha") != kernel_source_sha():
        return None, None
    return entry.get("dram_bytes_per_launch"), entry.get("note")


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_ours(args, dist: Dist):
    import torch

    from paper_2604_08374_gb300 import build as vga_build
    vga_build.build()
    import paper_2604_08374_gb300 as vga

    torch.cuda.set_device(dist.local_rank)
    dev = torch.device("cuda", dist.local_rank)
    obst = CONFIGS[args.config]["grid"]()
    t0 = time.perf_counter()
    g, cell_of_node = vga.vga_visibility_build(obst, order=args.order, return_cells=True)
    build_s = time.perf_counter() - t0
    N, E, B = g.n_nodes, g.n_edges, g.n_bytes
    tuned = None
    if args.autotune:
        t0 = time.perf_counter()
        tuned = vga.vga_autotune([g], p=args.p)
        tuned = {"entries": tuned, "seconds": round(time.perf_counter() - t0, 2)}
    ws = torch.empty(vga.hyperball_workspace_bytes(g, args.p), dtype=torch.uint8, device=dev)
    md = torch.empty(max(N, 1), dtype=torch.float64, device=dev)
    ball = torch.empty(max(N, 1), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    sharded = args.sharded and dist.world > 1
    if sharded:
        from paper_2604_08374_gb300.sharded import hyperball_run_sharded
        args.no_extras = True  # e2e, d = unlimited and the CPU leg are single-GPU measurements

    def step(d, union_mode=None, p=None, bits=None):
        if p is not None or bits is not None:  # sweep legs: other precision or register width, own workspace
            return vga.hyperball_run_dev(g, args.p if p is None else p, d, args.seed, md, ball, stream=stream,
                                         register_bits=0 if bits in (None, 8) else bits)
        if sharded and union_mode is None:
            with torch.cuda.stream(stream):
                return hyperball_run_sharded(g, args.p, d, args.seed, md, ball, slice_bytes=args.slice_bytes,
                                             warps_per_cta=args.warps, union_mode=args.union_mode,
                                             register_bits=0 if args.register_bits == 8 else args.register_bits,
                                             hub_lookups=args.hub_lookups, table_levels=args.table_levels,
                                             first_pass=args.first_pass, track_changes=args.track_changes,
                                             group_nodes=args.group_nodes)
        # a forced slice width or table scheme sizes its own workspace
        forced = args.slice_bytes or args.table_levels
        return vga.hyperball_run_dev(g, args.p, d, args.seed, md, ball, workspace=None if forced else ws,
                                     stream=stream,
                                     slice_bytes=args.slice_bytes, warps_per_cta=args.warps,
                                     union_mode=args.union_mode if union_mode is None else union_mode,
                                     register_bits=0 if args.register_bits == 8 else args.register_bits,
                                     hub_lookups=args.hub_lookups, table_levels=args.table_levels,
                                     l2_window=args.l2_window, first_pass=args.first_pass,
                                     track_changes=args.track_changes, group_nodes=args.group_nodes)

    for _ in range(args.warmup):
        step(args.d)

    # ---- timed region: K analyses, inputs resident ----
    vga.vga_profile_reset()
    vga.vga_profile_enable(True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    passes = 0
    for _ in range(args.steps):
        passes += step(args.d)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clock_info = clocks.stop()
    vga.vga_profile_enable(False)
    prof = vga.vga_profile_read()
    sec = e0.elapsed_time(e1) / 1e3
    if sharded:  # one analysis for the whole job: its edge unions once, the slowest rank's time
        units, sec_max = float(passes * E), dist.max(sec)
    else:
        units, sec_max = combine(passes * E, sec, dist)
    value = units / sec_max / 1e9

    # ---- roofline of the dominant kernel (the union pass) ----
    S = prof["slice_bytes"]
    mode = prof["union_mode"]
    avg_ms = prof["union_ms"] / max(prof["union_launches"], 1)
    gather_per_launch = prof["union_gather_bytes"] / max(prof["union_launches"], 1)
    hbm_per_launch = prof["union_hbm_bytes"] / max(prof["union_launches"], 1)
    l2_peak = vga.vga_bench_gather(N * S, S, 1_000_000_000 * 64 // S, consumer=1, stream=stream)
    loop_ceiling = vga.vga_bench_gather(N * S, S, 1_000_000_000 * 64 // S, consumer=0, stream=stream)
    # the bytes a union launch gathers from: the slice's table region (run-aware)
    # or the slice itself (per neighbour); streamed with coalesced loads, that
    # buffer gives the shape-independent L2 read ceiling
    src_bytes = N * S * (prof["table_rows"] if mode == 2 else 1)
    # an L2 figure needs an L2-resident buffer: at most 3/4 of the L2 (the
    # grouped union's region may be larger than the L2)
    l2_size = torch.cuda.get_device_properties(dev).L2_cache_size
    stream_bytes = max(min(src_bytes, l2_size * 3 // 4), 1 << 20)
    l2_stream = vga.vga_bench_gather(stream_bytes, S, 64_000_000_000 // S, consumer=2, stream=stream)
    achieved = gather_per_launch / (avg_ms / 1e3) / 1e9
    grouped = mode == 2 and args.group_nodes != 1
    kernel_name = (f"hb_union_groups_kernel<{S}>" if grouped else f"hb_union_runs_kernel<{S}>") if mode == 2 \
        else f"hb_union_kernel<{S}>"
    traffic, traffic_note = recorded_traffic(kernel_name, args.config)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak = max(l2_peak, l2_stream)
    # Sec. 8(d)'s definition of the gather bytes: every neighbour's register row,
    # E x S bytes per slice launch; the run-aware union gathers one table row per
    # run window instead, so against this definition it reads above any peak
    pn_achieved = E * S / (avg_ms / 1e3) / 1e9
    roofline = {
        "bound": "l2", "kernel": kernel_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak if peak else None,
        "traffic": traffic,
        "peak_source": ("the higher of two in-run L2 figures (MEASURED_PEAKS.json has no L2 peak): "
                        f"l2_stream, coalesced 16-byte L2-only loads streaming a {stream_bytes / 2**20:.0f} MiB "
                        "L2-resident buffer (the union's gather-source size, at most 3/4 of the L2) at full occupancy "
                        "(vga_bench_gather consumer=2), and gather_shape, hashed "
                        f"{S}-byte rows of an L2-resident {N * S / 2**20:.0f} MiB buffer with the union's own lane "
                        "mapping, load width and loads in flight (consumer=1).  The union's rows hit L1 about "
                        "45 % of the time (warps of one CTA take neighbouring nodes), the hashed rows never"),
        "l2_stream": {"value": l2_stream, "unit": "GB/s", "resident_bytes": stream_bytes,
                      "gather_source_bytes": src_bytes},
        "gather_shape": {"value": l2_peak, "unit": "GB/s", "resident_bytes": N * S},
        "frac_vs_l2_stream": achieved / l2_stream if l2_stream else None,
        "frac_vs_gather_shape": achieved / l2_peak if l2_peak else None,
        "frac_per_neighbour_definition": {
            "achieved": pn_achieved, "frac": pn_achieved / peak if peak else None, "unit": "GB/s",
            "definition": "E x slice_bytes bytes per slice launch (every neighbour's register row gathered, "
                          "B_L2 = E m per pass) over the same launch time; above 1 because the run-aware union "
                          "gathers one table row per window of a run of consecutive ids, not one per neighbour"},
        "union_loop_ceiling": {"value": loop_ceiling, "unit": "GB/s",
                               "what": "same microbenchmark folding with the union's bytewise max (no decode)"},
        "algorithmic_bytes_per_launch": gather_per_launch,
        "algorithmic_bytes_definition": (
            ("distinct table rows of the grouped lookup lists (groups of "
             f"{args.group_nodes or 4} consecutive nodes, each shared row gathered once) plus the split hubs' "
             "lookups, x slice_bytes, per slice launch (table build included in the timed launch)") if grouped else
            "range lookups x slice_bytes register-row gathers per slice launch (sparse-table build included in the "
            "timed launch); a lookup covers a run of consecutive neighbour ids" if mode == 2 else
            "E x slice_bytes neighbour-register gathers per slice launch"),
        "union_mode": mode,
        "avg_launch_ms": avg_ms, "launches_timed": prof["union_launches"],
        "hbm_term": {"algorithmic_bytes_per_launch": hbm_per_launch,
                     "achieved": hbm_per_launch / (avg_ms / 1e3) / 1e9, "peak": hbm_peak,
                     "frac": (hbm_per_launch / (avg_ms / 1e3) / 1e9 / hbm_peak) if hbm_peak else None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
    }
    if traffic_note:
        roofline["traffic_note"] = traffic_note
    # The bound of the per-neighbour method (one gather of every neighbour's
    # registers per edge, E x m bytes a pass, at the measured gather rate; the
    # CSR and register arrays at HBM peak): the run-aware union beats it by
    # gathering a table row per run instead.
    m_bytes = (1 << args.p) // (2 if args.register_bits == 4 else 1)
    t_l2 = E * m_bytes / (l2_peak * 1e9) if l2_peak else None
    t_hbm = (B + 8 * (N + 1) + 2 * N * m_bytes) / (hbm_peak * 1e9) if hbm_peak else None
    if t_l2 and t_hbm:
        per_nb = E / max(t_l2, t_hbm) / 1e9
        roofline["per_neighbour_roofline"] = {
            "geu_per_s": per_nb, "value_over_it": value / per_nb,
            "definition": "E / max((CSR + 8(N+1) + 2 N m) / hbm_gbs, E m / measured gather peak): the ceiling "
                          "of a union that gathers every neighbour's registers"}
    if prof["first_pass_launches"]:
        # pass 1 by the scatter of the nodes' hashes (one launch for all slices)
        fp_ms = prof["first_pass_ms"] / prof["first_pass_launches"]
        roofline["first_pass"] = {
            "kernel": "hb_first_pass_kernel", "launches_timed": prof["first_pass_launches"], "avg_launch_ms": fp_ms,
            "share_of_step": prof["first_pass_ms"] / (sec * 1e3) if sec > 0 else None,
            "edge_unions_per_s": E / (fp_ms / 1e3) / 1e9, "unit": "GEdge-unions/s",
            "what": "pass 1 of Eq. hll-union as a scatter: every counter holds only its own node, so each "
                    "neighbour's (register index, rho) is max-folded into shared-memory cells; no rows gathered"}
    union_share = (prof["union_ms"] + prof["first_pass_ms"]) / (sec * 1e3) if sec > 0 else None

    extras = {}
    if not args.no_extras:
        # ---- e2e: public C API with host buffers ----
        off_h, bytes_h, _ = g.copy_csr()
        off_pin = torch.empty(8 * len(off_h), dtype=torch.uint8, pin_memory=True)
        bytes_pin = torch.empty(max(len(bytes_h), 1), dtype=torch.uint8, pin_memory=True)
        off_np = off_pin.numpy().view(np.uint64)
        bytes_np = bytes_pin.numpy()[: len(bytes_h)]
        off_np[:] = off_h
        bytes_np[:] = bytes_h
        del bytes_h
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        e2e_passes = 0
        H, W = obst.shape
        for _ in range(args.steps):
            with vga.vga_graph_load(off_np, bytes_np) as g2:
                g2.set_cells(W, H, cell_of_node)  # the grid positions, as a caller holding the grid passes them
                _, _, it = vga.hyperball_run(g2, args.p, args.d, args.seed)
            e2e_passes += it
        s1.record()
        torch.cuda.synchronize()
        e2e_wall = time.perf_counter() - t0
        e2e_sec = s0.elapsed_time(s1) / 1e3
        e_units, e_sec = combine(e2e_passes * E, e2e_sec, dist)
        extras["e2e"] = {"value": e_units / e_sec / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * (N + 1) + B,
                         "d2h_bytes_per_step": 16 * N, "ms_per_step": 1e3 * e2e_sec / args.steps,
                         "wall_ms_per_step": 1e3 * e2e_wall / args.steps,
                         "calls": "vga_graph_load (pinned host CSR) + vga_graph_set_cells (the nodes' grid cells, host "
                                  "side) + hyperball_run (host outputs) + vga_graph_free"}
        del off_pin, bytes_pin
        # ---- unlimited depth, once ----
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        dinf_passes = step(0)
        f1.record(stream)
        torch.cuda.synchronize()
        extras["dinf"] = {"seconds": f0.elapsed_time(f1) / 1e3, "passes": dinf_passes,
                          "geu_per_s": dinf_passes * E / (f0.elapsed_time(f1) / 1e3) / 1e9}
        # ---- the other union variant, once, for comparison ----
        other = 1 if mode == 2 else 2
        step(args.d, union_mode=other)
        f0.record(stream)
        o_passes = step(args.d, union_mode=other)
        f1.record(stream)
        torch.cuda.synchronize()
        extras["other_union_mode"] = {"union_mode": other, "seconds": f0.elapsed_time(f1) / 1e3,
                                      "geu_per_s": o_passes * E / (f0.elapsed_time(f1) / 1e3) / 1e9}
        # ---- sweeps of the city configuration: p = 8 and 12, d = 10, and the
        #      paper's packed 4-bit registers (rho clamped to 15) ----
        sweep = []
        for (sp, sd, sb) in ((8, args.d, 8), (12, args.d, 8), (args.p, 10, 8), (args.p, args.d, 4)):
            step(sd, p=sp, bits=sb)
            if sb == 4:  # the packed format's union launches against the same L2 ceilings
                vga.vga_profile_reset()
                vga.vga_profile_enable(True)
            f0.record(stream)
            s_passes = step(sd, p=sp, bits=sb)
            f1.record(stream)
            torch.cuda.synchronize()
            sec_s = f0.elapsed_time(f1) / 1e3
            entry = {"p": sp, "d": sd, "register_bits": sb, "seconds": sec_s, "passes": s_passes,
                     "geu_per_s": s_passes * E / sec_s / 1e9}
            if sb == 4:
                vga.vga_profile_enable(False)
                p4 = vga.vga_profile_read()
                if p4["union_launches"]:
                    ms4 = p4["union_ms"] / p4["union_launches"]
                    ach4 = p4["union_gather_bytes"] / p4["union_launches"] / (ms4 / 1e3) / 1e9
                    entry["union"] = {"slice_bytes": p4["slice_bytes"], "launches_timed": p4["union_launches"],
                                      "avg_launch_ms": ms4, "achieved_gbs": ach4,
                                      "frac_vs_l2_stream": ach4 / l2_stream, "frac_vs_gather_shape": ach4 / l2_peak,
                                      "what": "distinct table rows x slice bytes per launch over the launch time "
                                              "(a 128-byte row holds 256 packed registers)"}
            sweep.append(entry)
        # register shards (the multi-GPU split) run in lockstep on this one GPU: the same
        # union work as one run plus the per-pass partial sums and their estimate, so the
        # time over the unsharded run is the split's compute overhead (no interconnect)
        if not sharded:
            from paper_2604_08374_gb300.sharded import hyperball_run_sharded_local
            hyperball_run_sharded_local(g, args.p, args.d, args.seed, 2, md, ball, stream=stream)
            f0.record(stream)
            sh_passes = hyperball_run_sharded_local(g, args.p, args.d, args.seed, 2, md, ball, stream=stream)
            f1.record(stream)
            torch.cuda.synchronize()
            sec_sh = f0.elapsed_time(f1) / 1e3
            extras["shards_local"] = {"n_shards": 2, "seconds": sec_sh, "passes": sh_passes,
                                      "unsharded_seconds": sec_max / args.steps,
                                      "overhead": sec_sh / (sec_max / args.steps) - 1.0}
        # the paper's optional Hilbert numbering (Sec. 3.2): the same grid, its own graph
        if args.order == "raster":
            gh = vga.vga_visibility_build(obst, order="hilbert")
            mdh = torch.empty(max(gh.n_nodes, 1), dtype=torch.float64, device=dev)
            vga.hyperball_run_dev(gh, args.p, args.d, args.seed, mdh, None, stream=stream)
            f0.record(stream)
            h_passes = vga.hyperball_run_dev(gh, args.p, args.d, args.seed, mdh, None, stream=stream)
            f1.record(stream)
            torch.cuda.synchronize()
            sec_h = f0.elapsed_time(f1) / 1e3
            sweep.append({"order": "hilbert", "p": args.p, "d": args.d, "csr_bytes": gh.n_bytes, "seconds": sec_h,
                          "passes": h_passes, "geu_per_s": h_passes * gh.n_edges / sec_h / 1e9})
            gh.free()
        extras["sweep"] = sweep
        if dist.rank == 0 and dist.world == 1:
            extras["cpu_baseline"] = cpu_baseline(obst, args)
            extras["cpu_baseline"]["full_analysis_medium"] = full_analysis_medium(vga, torch, stream)
            if not args.no_serve:
                # the batched and served workloads, as records of this same run
                extras["batch"] = batch_leg(vga, torch, args.steps)
                extras["serve"] = serve_leg(vga, torch, args.serve_requests, args.serve_pool, args.solo_nodes,
                                            args.lane_priority, args.batched_share)
        # the GPU visibility builder (run once before the timed region) beside the oracle's
        extras["builder"] = {"gpu_seconds": build_s, "pair_tests": N * (N - 1) // 2,
                             "pair_tests_per_s": N * (N - 1) / 2 / build_s,
                             "what": "vga_visibility_build: main component on the host, then each source's "
                                     "8 octants swept column by column on the device with exact slope intervals, "
                                     "lists counted and LEB128-encoded in two passes; pair_tests = the N(N-1)/2 "
                                     "pairs it decides"}
        if "cpu_baseline" in extras:
            cb = extras["cpu_baseline"]["builder"]
            extras["builder"]["cpu_oracle_pair_tests_per_s"] = cb["pair_tests_per_s"]
            extras["builder"]["cpu_oracle_cores"] = extras["cpu_baseline"]["cores"]

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": CONFIGS[args.config]["name"], "p": args.p, "d": args.d, "seed": args.seed,
                       "N": N, "E": E, "csr_bytes": B, "slice_bytes": S, "union_mode": mode, "order": args.order,
                       "register_bits": args.register_bits, "table_levels": args.table_levels or "auto",
                       "l2_window": args.l2_window, "group_nodes": args.group_nodes or ("auto (4)" if mode == 2 else None),
                       "first_pass": {0: "auto", 1: "gather", 2: "scatter"}[args.first_pass],
                       "track_changes": {0: "auto", 1: "off", 2: "every pass"}[args.track_changes],
                       "autotune": tuned,
                       "parallelism": f"register shards x{dist.world}" if sharded else f"replicas x{dist.world}",
                       "l2": "inputs larger than L2 (compressed CSR > 129 MB), no flush",
                       "graph_build_seconds": build_s},
            "roofline": roofline, "gpu_launches": prof["kernel_launches"], "union_time_share": union_share,
            "clocks": clock_info, "passes_per_step": passes / args.steps, "context": PAPER_CONTEXT}
    line.update(extras)
    if "e2e" not in line:
        line["e2e"] = None
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    g.free()


# ----------------------------------------------------------------------------
# batched and served workloads (our arm only)
# ----------------------------------------------------------------------------

def _percentile(xs, q):
    return float(np.percentile(np.asarray(xs, np.float64), q)) if len(xs) else None


def batch_leg(vga, torch, steps: int, count: int = 256, autotune: bool = False) -> dict:
    """256 graphs of 1k-30k cells, p in {8,10,12}, d in {3, unlimited}: one
    hyperball_run_batch call against the same analyses run one at a time with
    hyperball_run_dev (best of two rounds each way)."""
    specs = workloads.batch(count, seed=0)
    t0 = time.perf_counter()
    graphs = [vga.vga_visibility_build(sp["grid"]) for sp in specs]
    build_s = time.perf_counter() - t0
    jobs = [dict(graph=g, p=sp["p"], d=sp["d"], seed=k, conv_mode=0,
                 mean_depth=torch.empty(max(g.n_nodes, 1), dtype=torch.float64, device="cuda"),
                 ball=torch.empty(max(g.n_nodes, 1), dtype=torch.float64, device="cuda"))
            for k, (g, sp) in enumerate(zip(graphs, specs))]
    nodes = [g.n_nodes for g in graphs]
    edges = [g.n_edges for g in graphs]
    tuned = None
    if autotune:
        t0 = time.perf_counter()
        tuned = {"entries": vga.vga_autotune(graphs, p=10), "seconds": round(time.perf_counter() - t0, 2)}
    # one at a time (each with a reused workspace); the first round warms caches and lookup lists
    ws_single = torch.empty(max(vga.hyperball_workspace_bytes(j["graph"], j["p"]) for j in jobs), dtype=torch.uint8,
                            device="cuda")
    single_md, single = [], []
    for rep in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in jobs:
            md = torch.empty_like(j["mean_depth"])
            vga.hyperball_run_dev(j["graph"], j["p"], j["d"], j["seed"], md, None, workspace=ws_single)
            if rep == 2:
                single_md.append(md)
        torch.cuda.synchronize()
        if rep:
            single.append(time.perf_counter() - t0)
    # batched: warm-up, then timed, in CUDA-graph mode and host-driven mode
    ws = torch.empty(vga.hyperball_batch_workspace_bytes(jobs), dtype=torch.uint8, device="cuda")
    vga.hyperball_run_batch(jobs, workspace=ws, use_graph=True)
    timings = {}
    its = []
    for mode in (True, False):
        reps = []
        for _ in range(max(2, steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its = vga.hyperball_run_batch(jobs, workspace=ws, use_graph=mode)
            torch.cuda.synchronize()
            reps.append(time.perf_counter() - t0)
        timings["graph" if mode else "host"] = min(reps)
    identical = all(torch.equal(torch.nan_to_num(j["mean_depth"][: j["graph"].n_nodes], nan=-1.0),
                                torch.nan_to_num(m[: j["graph"].n_nodes], nan=-1.0))
                    for j, m in zip(jobs, single_md))
    n = len(jobs)
    best = min(timings.values())
    single_s = min(single)
    out = {"metric": "batched analyses/s (256 graphs of 1k-30k cells, p in {8,10,12}, d in {3, unlimited})",
           "value": n / best, "unit": "analyses/s",
           "config": {"workload": f"{n} medium-style grids, free cells log-uniform 1k-30k, per-graph seeds",
                      "nodes_total": int(sum(nodes)), "edges_total": int(sum(edges)),
                      "graph_build_seconds": round(build_s, 3), "autotune": tuned},
           "batched_seconds": best, "batched_graph_loop_seconds": timings["graph"],
           "batched_host_loop_seconds": timings["host"],
           "one_at_a_time_seconds": single_s, "one_at_a_time_analyses_per_s": n / single_s,
           "speedup_vs_one_at_a_time": single_s / best,
           "passes_total": int(sum(its)), "results_identical_to_one_at_a_time": bool(identical),
           "timing": "wall clock around each call with device synchronisation, best of runs; batched_seconds is "
                     "the faster of the CUDA-graph and host-driven pass loops"}
    for g in graphs:
        g.free()
    return out


def serve_leg(vga, torch, R: int, pool_size: int = 64, solo_nodes: int = 0, lane_priority: int = 0,
              batched_share: int = 0) -> dict:
    """Poisson (graph, p, d) requests over a resident pool of graphs at 0.5x,
    0.9x and 1.5x the measured one-at-a-time capacity, through vga_server
    (150 GiB budget), against (a) the measured one-at-a-time loop (the plain
    public call per request, in arrival order, each started at its arrival or
    when the previous one ends) and (b) an idealised FIFO replay of each
    request's solo service time (measured once per distinct analysis)."""
    import threading

    t0 = time.perf_counter()
    pool = [vga.vga_visibility_build(g) for g in workloads.serve_pool(pool_size, seed=0)]
    build_s = time.perf_counter() - t0
    base = workloads.serve_requests(R, len(pool), rate=1.0, seed=1)
    # solo service time of every distinct (graph, p, d); first warm every graph's lookup lists
    for g in pool:
        vga.hyperball_run(g, 8, 1, 0)
    solo = {}
    for (_, gi, p, d) in base:
        if (gi, p, d) in solo:
            continue
        g = pool[gi]
        md = torch.empty(max(g.n_nodes, 1), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        vga.hyperball_run_dev(g, p, d, 0, md, None)
        torch.cuda.synchronize()
        solo[(gi, p, d)] = time.perf_counter() - t1
    service = [solo[(gi, p, d)] for (_, gi, p, d) in base]
    capacity = R / sum(service)
    loads = []
    for f in (0.5, 0.9, 1.5):
        rate = f * capacity
        arrivals = [a / rate for (a, _, _, _) in base]
        free_at, lat_single = 0.0, []
        for a, s_k in zip(arrivals, service):
            start = max(a, free_at)
            free_at = start + s_k
            lat_single.append(free_at - a)
        single_makespan = free_at - arrivals[0]
        lat_fifo, t0f = [], time.perf_counter()
        t_done = t0f
        for k, (a, (_, gi, p, d)) in enumerate(zip(arrivals, base)):
            delay = t0f + a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            vga.hyperball_run(pool[gi], p, d, k)
            t_done = time.perf_counter()
            lat_fifo.append(t_done - (t0f + a))
        fifo_makespan = t_done - (t0f + arrivals[0])
        with vga.Server(hbm_budget_bytes=150 << 30, solo_nodes=solo_nodes, lane_priority=lane_priority,
                        batched_share=batched_share) as srv:
            ids = [None] * R
            submit_t = [0.0] * R
            t_start = time.perf_counter()

            def submitter():
                for k, (a, (_, gi, p, d)) in enumerate(zip(arrivals, base)):
                    delay = t_start + a - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    submit_t[k] = time.perf_counter()
                    ids[k] = srv.submit(pool[gi], p, d, k)

            th = threading.Thread(target=submitter)
            th.start()
            lat, done_t = [], []
            for k in range(R):
                while ids[k] is None:
                    time.sleep(0.0005)
                out = srv.wait(ids[k], timeout_s=600)
                lat.append(out["latency_s"])
                done_t.append(submit_t[k] + out["latency_s"])
            th.join()
            st = srv.stats()
        served_makespan = max(done_t) - submit_t[0]
        served = {"analyses_per_s": R / served_makespan, "p50_s": _percentile(lat, 50),
                  "p99_s": _percentile(lat, 99), "batched_peak": st["batched_peak"],
                  "budget_peak_bytes": st["budget_peak"]}
        measured = {"analyses_per_s": R / fifo_makespan, "p50_s": _percentile(lat_fifo, 50),
                    "p99_s": _percentile(lat_fifo, 99)}
        loads.append({"offered_load": f, "rate_per_s": rate, "served": served,
                      "one_at_a_time_measured": measured,
                      "one_at_a_time_ideal": {"analyses_per_s": R / single_makespan,
                                              "p50_s": _percentile(lat_single, 50),
                                              "p99_s": _percentile(lat_single, 99)},
                      "served_beats_measured": {
                          "p50": served["p50_s"] <= measured["p50_s"], "p99": served["p99_s"] <= measured["p99_s"],
                          "throughput": served["analyses_per_s"] >= measured["analyses_per_s"]}})
    out = {"metric": "served analyses/s and p50/p99 latency (Poisson requests, pool of 64 graphs 1k-236k cells)",
           "value": loads[-1]["served"]["analyses_per_s"], "unit": "analyses/s",
           "config": {"workload": f"pool of {len(pool)} medium-style grids, free cells log-uniform 1k-236k; "
                                  f"{R} requests per load, p in {{8,10,12}}, d in {{3,5,unlimited}}",
                      "pool_nodes_total": int(sum(g.n_nodes for g in pool)),
                      "pool_edges_total": int(sum(g.n_edges for g in pool)),
                      "hbm_budget_bytes": 150 << 30, "graph_build_seconds": round(build_s, 3),
                      "lane_priority": lane_priority, "solo_nodes": solo_nodes or 32768,
                      "batched_share": batched_share, "distinct_analyses_timed_solo": len(solo)},
           "one_at_a_time_capacity_per_s": capacity, "loads": loads,
           "what": "one_at_a_time_measured: hyperball_run (host outputs) per request in arrival order on one "
                   "thread, timed from each arrival; one_at_a_time_ideal: FIFO replay of each request's solo "
                   "service time with no host overhead"}
    for g in pool:
        g.free()
    return out


def run_batch_mode(args, dist):
    import torch

    from paper_2604_08374_gb300 import build as vga_build
    vga_build.build()
    import paper_2604_08374_gb300 as vga
    torch.cuda.set_device(dist.local_rank)
    line = batch_leg(vga, torch, args.steps, args.batch_count, args.autotune)
    line.update({"n_gpus": dist.world, "higher_is_better": True, "data": "synthetic", "dtype": "u8"})
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def run_serve_mode(args, dist):
    import torch

    from paper_2604_08374_gb300 import build as vga_build
    vga_build.build()
    import paper_2604_08374_gb300 as vga
    torch.cuda.set_device(dist.local_rank)
    line = serve_leg(vga, torch, args.serve_requests, args.serve_pool, args.solo_nodes, args.lane_priority,
                     args.batched_share)
    line.update({"n_gpus": dist.world, "higher_is_better": True, "data": "synthetic", "dtype": "u8"})
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    dist = Dist(args.backend)
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.mode == "batch":
            run_batch_mode(args, dist)
        elif args.mode == "serve":
            run_serve_mode(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
