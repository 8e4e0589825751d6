#!/usr/bin/env python
"""Benchmark of the tile-wise LISI / augLISI maps (arxiv 2501.10653) on GB300.

Workload (the paper's Section 3 shape): N = 2048, N_T = 64 (1024 tiles), FP32
storage, synthetic radio-sky pairs (33 Gaussian-beam sources, sigma 2e-4
noise, 1e-4 diffuse ripple, the 5 faintest sources dropped in epoch 2).  One
step = one ``iqa_both`` call through the C-ABI: both maps from a single read of
each pixel of one pair.  Inputs rotate over a pool of distinct pairs larger
than twice the L2 cache, so every step reads its pixels from HBM.

Prints ONE JSON line (rank 0).  ``value`` is the whole-job HBM throughput
(algorithmic bytes 2 N^2 * 4 per pair) over the K timed steps; ``e2e`` is the
same metric through ``iqa_both_host`` with page-locked host buffers (uploads
and map read-back inside the timed region); ``cpu_baseline`` times the FP64
oracle on the host cores on a bounded sample.

``--impl reference`` times the FP64 CPU oracle itself on the same workload
(each step a bounded band of tile rows) and prints its own line.

Multi-GPU: one process per GPU (torchrun); each rank streams its own pairs
(independent replicas, no data-path collective), and the timing is the max
over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("LISI/augLISI HBM GB/s (% of peak) and pairs/s at N=2048,N_T=64; "
          "served p50/p99 ms")
N_IMG = 2048
N_TILE = 64
PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.5e-6}
PAPER_H100 = {"lisi_kernel_ms": 0.101, "auglisi_kernel_ms": 0.091,
              "hardware": "H100", "note": "context only (another machine)"}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pool", type=int, default=10,
                    help="distinct device pairs the steps rotate over")
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="bound on the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------
# distributed plumbing (one process per GPU)

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------
# measured peaks and clocks

def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


class ClockSampler:
    """nvidia-smi samples every 200 ms while running (SM clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on the host cores

def cpu_baseline(x, y, seconds):
    import oracle
    orc = oracle.Oracle()
    threads = (os.cpu_count() or 1) if orc.has_openmp else 1
    N = x.shape[0]
    T = N // N_TILE
    # a bounded sample: bands of whole tile rows, repeated until `seconds`
    rows_per_call = max(1, T // 8)
    done_px, t0, calls = 0, time.perf_counter(), 0
    while True:
        r0 = (calls * rows_per_call) % T
        r1 = min(T, r0 + rows_per_call)
        tiles = np.arange(r0 * T, r1 * T)
        orc.tile_sums(x, y, N_TILE, PARAMS["C1"], tiles=tiles, threads=threads)
        done_px += (r1 - r0) * N_TILE * N
        calls += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    gbs = done_px * 8 / el / 1e9
    return {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": "%d tile-row bands (%d x %d px each) of one N=2048 FP32 pair, "
                      "N_T=64, %.1f s of FP64 oracle work" % (calls, rows_per_call * N_TILE,
                                                             N, el),
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


# --------------------------------------------------------------------------
# our implementation

def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)

    from paper_2501_10653_gb300 import build as lib_build
    if rank == 0 or world == 1:
        lib_build.build()
    barrier(world)
    from paper_2501_10653_gb300 import iqa, synth

    N, NT = N_IMG, N_TILE
    T = N // NT
    pair_bytes = 2 * N * N * 4
    ctx = iqa.iqa_create(local, 0)
    params = iqa.iqa_params(PARAMS["C1"], PARAMS["C2"], PARAMS["C"], PARAMS["D"])

    # distinct pairs per rank (independent replicas)
    host_pairs = [synth.paper_pair(pair_index=rank * args.pool + i) for i in range(args.pool)]
    dx = [torch.from_numpy(x).to(dev) for x, _ in host_pairs]
    dy = [torch.from_numpy(y).to(dev) for _, y in host_pairs]
    lisi = [torch.empty(T * T, device=dev) for _ in range(args.pool)]
    aug = [torch.empty(T * T, device=dev) for _ in range(args.pool)]
    stream = torch.cuda.Stream(device=dev)
    cfg = iqa.iqa_get_config(ctx, iqa.IQA_F32, N, NT, iqa.MAPS_BOTH).as_dict()

    def step(i, st):
        j = i % args.pool
        iqa.iqa_both(ctx, dx[j], dy[j], iqa.IQA_F32, N, NT, params, lisi[j], aug[j],
                     None, st)

    clocks = ClockSampler(local)
    clocks.start()
    with torch.cuda.stream(stream):
        for i in range(max(3, args.warmup)):
            step(i, stream)
    torch.cuda.synchronize()

    # the timed K steps are replayed from a CUDA graph of G steps so that no
    # host-side launch cost enters the device timing
    K = max(1, args.steps)
    G = min(K, 10 * args.pool)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for i in range(G):
            step(i, stream)
    tail = K % G
    graph_tail = None
    if tail:
        graph_tail = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_tail, stream=stream):
            for i in range(tail):
                step(i, stream)
    torch.cuda.synchronize()

    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(K // G):
            graph.replay()
        if graph_tail is not None:
            graph_tail.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    dev_ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    t_max_ms = max_over_ranks(dev_ms, world, dev)

    # per-launch duration (events around single launches, a GPU-side delay
    # ahead of each so the host call cost stays outside the events)
    single = []
    for i in range(20):
        with torch.cuda.stream(stream):
            torch.cuda._sleep(200000)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            step(i + 3, stream)
            a1.record(stream)
        torch.cuda.synchronize()
        single.append(a0.elapsed_time(a1) * 1e3)
    single_us = float(np.median(single[3:]))

    # end to end through the host-buffer entry point (page-locked buffers)
    hx = [torch.from_numpy(x).pin_memory() for x, _ in host_pairs[:4]]
    hy = [torch.from_numpy(y).pin_memory() for _, y in host_pairs[:4]]
    hl = np.empty(T * T, np.float32)
    ha = np.empty(T * T, np.float32)
    for i in range(3):
        iqa.iqa_both_host(ctx, hx[i % 4], hy[i % 4], iqa.IQA_F32, N, NT, params, hl, ha)
    barrier(world)
    t0 = time.perf_counter()
    E = max(1, args.e2e_steps)
    for i in range(E):
        iqa.iqa_both_host(ctx, hx[i % 4], hy[i % 4], iqa.IQA_F32, N, NT, params, hl, ha)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    assert np.all(np.isfinite(hl)) and np.all(np.isfinite(ha))

    total_bytes = sum_over_ranks(K * pair_bytes, world, dev)
    value = total_bytes / (t_max_ms * 1e-3) / 1e9
    peak, peak_src = measured_peak()
    per_launch_us = dev_ms * 1e3 / K
    achieved = pair_bytes / (per_launch_us * 1e-6) / 1e9
    e2e_value = sum_over_ranks(E * pair_bytes, world, dev) / e2e_s / 1e9

    result = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(host_pairs[0][0], host_pairs[0][1], args.cpu_seconds)
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s",
            "n_gpus": world, "steps": K, "warmup": max(3, args.warmup),
            "ms_per_step": round(t_max_ms / K, 6), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian-beam radio skies, no dataset)",
            "config": {"workload": "paper-scale pair N=2048 N_T=64 FP32, LISI+augLISI "
                                   "in one pass", "N": N, "N_T": NT, "tiles": T * T,
                       "pool_pairs": args.pool,
                       "l2": "inputs larger than L2: steps rotate over %d distinct pairs "
                             "(%d MB)" % (args.pool, args.pool * pair_bytes // 2 ** 20),
                       "params": PARAMS, "launch": cfg,
                       "timing": "CUDA events around K steps replayed from a CUDA graph",
                       "parallelism": "replicas x%d" % world},
            "pct_of_peak": round(100 * value / world / peak, 2),
            "pairs_per_s": round(value * 1e9 / pair_bytes, 1),
            "pixel_pairs_per_s": round(value * 1e9 / 8, 1),
            "kernel_us_per_pair": round(per_launch_us, 3),
            "single_launch_us": round(single_us, 3),
            "clocks": clk,
            "e2e": {"value": round(e2e_value, 2), "unit": "GB/s",
                    "h2d_bytes_per_step": pair_bytes,
                    "d2h_bytes_per_step": 2 * T * T * 4,
                    "ms_per_step": round(e2e_s * 1e3 / E, 4),
                    "api": "iqa_both_host, page-locked host buffers"},
            "gpu_launches": K,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": None, "peak_source": peak_src,
                         "kernel": "iqa_tiles_kernel f32 threads=%d ilp=%d tiles_across=%d "
                                   "split=%d" % (cfg["threads"], cfg["ilp"],
                                                 cfg["tiles_across"], cfg["split"])},
            "cpu_baseline": cpu,
            "paper_context": PAPER_H100,
        }
    iqa.iqa_destroy(ctx)
    return result


# --------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the same workload

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    from paper_2501_10653_gb300 import synth
    orc = oracle.Oracle()
    threads = (os.cpu_count() or 1) if orc.has_openmp else 1
    x, y = synth.paper_pair()
    N, NT = N_IMG, N_TILE
    T = N // NT
    K = max(1, args.steps)
    W = max(3, args.warmup)
    # per-step sample: a band of whole tile rows, sized so that the whole run
    # stays within about two minutes
    t0 = time.perf_counter()
    orc.tile_sums(x, y, NT, PARAMS["C1"], tiles=np.arange(T), threads=threads)
    row_s = max(1e-4, time.perf_counter() - t0)
    budget = 120.0 / (K + min(W, 10))
    rows = int(max(1, min(T, budget / row_s)))
    tiles = np.arange(rows * T)
    for _ in range(min(W, 10)):
        orc.tile_sums(x, y, NT, PARAMS["C1"], tiles=tiles, threads=threads)
    t0 = time.perf_counter()
    for _ in range(K):
        orc.tile_sums(x, y, NT, PARAMS["C1"], tiles=tiles, threads=threads)
    el = time.perf_counter() - t0
    step_bytes = rows * NT * N * 8
    value = K * step_bytes / el / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": world, "steps": K, "warmup": min(W, 10),
        "ms_per_step": round(el * 1e3 / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian-beam radio skies, no dataset)",
        "config": {"workload": "paper-scale pair N=2048 N_T=64 FP32, LISI+augLISI "
                               "in one pass", "N": N, "N_T": NT, "params": PARAMS,
                   "sample_tile_rows": rows, "parallelism": "host cores"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads,
                         "kind": "oracle",
                         "sample": "%d of %d tile rows of one N=2048 pair per step" % (rows, T)},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        res = run_reference(args)
    else:
        res = run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
