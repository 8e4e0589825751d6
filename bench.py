#!/usr/bin/env python
"""Benchmark of the tile-wise LISI / augLISI maps (arxiv 2501.10653) on GB300.

Workload (the paper's Section 3 shape): N = 2048, N_T = 64 (1024 tiles), FP32
storage, synthetic radio-sky pairs (33 Gaussian-beam sources, sigma 2e-4
noise, 1e-4 diffuse ripple, the 5 faintest sources dropped in epoch 2).  One
step = one persistent launch (a replayed CUDA graph of ``iqa_plan_launch``)
that computes both maps of B distinct such pairs from a single read of each
pixel; B pairs are 33.5 MB each, far larger than the L2 cache, so every step
reads its pixels from HBM.  The one-pair-per-launch form (``iqa_both``) is
timed beside it.

Prints ONE JSON line (rank 0).  ``value`` is the whole-job HBM throughput
(algorithmic bytes 2 N^2 * 4 per pair) over the K timed steps; ``e2e`` is the
same metric through ``iqa_both_host_many`` with page-locked host buffers
(uploads and map read-back inside the timed region); ``cpu_baseline`` times the FP64
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
PAPER_NT_SWEEP = (16, 32, 64, 128, 256)
PAPER_N_SWEEP = (512, 1024, 2048, 4096, 8192)

# DRAM traffic of the timed kernel from one ncu capture of the timed launch
# itself (its summary and command are under profiles/, named for this kernel
# and workload):
# dram__bytes_read.sum + dram__bytes_write.sum of the first launch inside the
# headline_timed NVTX range, 32 pairs.  Valid only for the kernel sources it was
# taken on: `traffic` is reported as null when their hash no longer matches.
PROFILED_TRAFFIC = {
    "sources": ["paper_2501_10653_gb300/csrc/iqa_device.cuh",
                "paper_2501_10653_gb300/csrc/iqa_stream.cuh",
                "paper_2501_10653_gb300/csrc/iqa_stream_f32.cu",
                "paper_2501_10653_gb300/csrc/iqa_stream_host.cpp"],
    "sha256": "ca0faa968ff0e8c658394320d0e5cc3f7330f8f66bfa183c706e75e8a5af6b1f",
    "bytes_per_launch": 1073832704 + 3502336,
    "pairs_per_launch": 32,
    "capture": "the timed launch itself (first launch in the headline_timed NVTX range, "
               "32 pairs, 456 CTAs of 160 threads)",
}
# the workload both arms measure (the reference arm times a bounded sample)
WORKLOAD = ("paper-scale pairs N=2048 N_T=64 FP32, LISI+augLISI in one pass, distinct "
            "pairs resident in memory")
PAPER_H100 = {"lisi_kernel_ms": 0.101, "auglisi_kernel_ms": 0.091,
              "hardware": "H100", "note": "context only (another machine)"}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=32,
                    help="distinct N=2048 pairs per step (one persistent launch)")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="bound on the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-merge", action="store_true",
                    help="skip the Eq. 3 / Eq. 4 merge report")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the N=8192 FP32/FP16/BF16 precision and throughput report")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the 64-pair mixed-size batch report")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served Poisson trace (0: skip serving)")
    ap.add_argument("--precision-batch", type=int, default=16,
                    help="N=8192 pairs per launch in the precision throughput report")
    ap.add_argument("--tune-iters", type=int, default=10,
                    help="launches per autotuner candidate (0: keep the default shape)")
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

def profiled_traffic(pairs_per_launch):
    import hashlib
    h = hashlib.sha256()
    try:
        for f in PROFILED_TRAFFIC["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    if h.hexdigest() != PROFILED_TRAFFIC["sha256"]:
        return None
    if pairs_per_launch == PROFILED_TRAFFIC["pairs_per_launch"]:
        return PROFILED_TRAFFIC["bytes_per_launch"]
    # another batch size: scaled by pairs (traffic grows in proportion)
    return int(round(PROFILED_TRAFFIC["bytes_per_launch"] * pairs_per_launch /
                     PROFILED_TRAFFIC["pairs_per_launch"]))


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

def _oracle_rate(orc, x, y, seconds, threads):
    """FP64 oracle throughput (GB/s of FP32 pair bytes) over bands of whole
    tile rows of one pair, repeated until `seconds` have passed."""
    N = x.shape[0]
    T = N // N_TILE
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
    return done_px * 8 / el / 1e9, calls, rows_per_call, el


def cpu_baseline(x, y, seconds):
    import oracle
    orc = oracle.Oracle()
    threads = (os.cpu_count() or 1) if orc.has_openmp else 1
    N = x.shape[0]
    gbs, calls, rows_per_call, el = _oracle_rate(orc, x, y, seconds, threads)
    one, _, _, el1 = _oracle_rate(orc, x, y, max(1.0, seconds / 4), 1)
    return {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": "%d tile-row bands (%d x %d px each) of one N=2048 FP32 pair, "
                      "N_T=64, %.1f s of FP64 oracle work" % (calls, rows_per_call * N_TILE,
                                                             N, el),
            "single_thread_value": round(one, 4),
            "single_thread_seconds": round(el1, 1),
            "cpu": _cpu_model()}


def _widen16(a):
    if a.dtype == np.uint16:
        return (a.astype(np.uint32) << 16).view(np.float32)
    return a.astype(np.float32)


def precision_errors(prec_maps, prec):
    """CPU-baseline leg, outside every timed region: pair 0 of the precision
    workload, as the timed FP32 / FP16 / BF16 launches computed it, against
    the FP64 oracle -- on the stored (rounded) pixels (accumulation error) and
    on the FP32 originals (storage + accumulation error) -- with the stated
    storage bound (oracle.storage_bound, from the originals alone) checked on
    every tile."""
    import oracle
    from oracle import storage_bound
    orc = oracle.Oracle()
    threads = (os.cpu_count() or 1) if orc.has_openmp else 1
    x32, y32, maps = prec_maps
    NT = 64
    C1, C2, C, D = PARAMS["C1"], PARAMS["C2"], PARAMS["C"], PARAMS["D"]
    ol, oa, osum = orc.maps(x32, y32, NT, C1, C2, C, D, threads=threads)
    ol, oa = ol.ravel(), oa.ravel()
    r32 = osum[:, 1] / (osum[:, 2] + osum[:, 3] + C)
    for name, (x, y, gl, ga) in maps.items():
        gl = gl.astype(np.float64).ravel()
        ga = ga.astype(np.float64).ravel()
        rl, ra, rsum = orc.maps(_widen16(x), _widen16(y), NT, C1, C2, C, D, threads=threads)
        rl, ra = rl.ravel(), ra.ravel()
        rr = rsum[:, 1] / (rsum[:, 2] + rsum[:, 3] + C)
        nz = rl > 0
        acc_l = np.abs(gl - rl)[nz] / rl[nz]
        acc_a = np.abs(ga - ra) / np.maximum(np.abs(ra), rr)
        nz32 = ol > 0
        st_l = np.abs(gl - ol)[nz32] / ol[nz32]
        st_a = np.abs(ga - oa) / np.maximum(np.abs(oa), r32)
        lb, ab, _, _ = storage_bound.tile_bounds(x32, y32, NT, name, C1, C2, C, D)
        ok = bool(np.all(np.abs(gl - ol) <= lb + 1e-5 * np.abs(rl)) and
                  np.all(np.abs(ga - oa) <= ab + 1e-5 * np.maximum(np.abs(ra), rr)))
        prec[name].update({
            "acc_err_lisi_rel_max": float("%.3g" % acc_l.max()),
            "acc_err_aug_max": float("%.3g" % acc_a.max()),
            "storage_err_lisi_rel_median": float("%.3g" % np.median(st_l)),
            "storage_err_lisi_rel_max": float("%.3g" % st_l.max()),
            "storage_err_aug_max": float("%.3g" % st_a.max()),
            "stated_bound_lisi_rel_max": float("%.3g" % np.max(lb[nz32] / ol[nz32])),
            "stated_bound_aug_max": float("%.3g" % np.max(ab / np.maximum(np.abs(oa), r32))),
            "within_stated_bound_every_tile": ok,
        })
    prec["errors"] = ("pair 0 of the timed launches against the FP64 oracle: acc_err on the "
                      "stored pixels (bar 1e-5), storage_err on the FP32 originals; the "
                      "stated storage bound (computed from the originals alone) plus the "
                      "1e-5 accumulation bar checked on all %d tiles" % ol.size)


def small_pair_errors(small, orc_threads=None):
    """CPU-baseline leg: the small pair's GPU maps against the FP64 oracle."""
    import oracle
    orc = oracle.Oracle()
    threads = orc_threads or ((os.cpu_count() or 1) if orc.has_openmp else 1)
    x, y, gl, ga = small.pop("_maps")
    C1, C2, C, D = PARAMS["C1"], PARAMS["C2"], PARAMS["C"], PARAMS["D"]
    ol, oa, osum = orc.maps(x, y, 64, C1, C2, C, D, threads=threads)
    ol, oa = ol.ravel(), oa.ravel()
    r = osum[:, 1] / (osum[:, 2] + osum[:, 3] + C)
    small["max_rel_err_lisi"] = float("%.3g" % np.max(np.abs(gl - ol) / ol))
    small["max_rel_err_aug"] = float("%.3g" % np.max(np.abs(ga - oa) /
                                                      np.maximum(np.abs(oa), r)))


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

def _pool_pairs(rank, count):
    from paper_2501_10653_gb300 import synth
    return [synth.paper_pair(pair_index=rank * count + i) for i in range(count)]


def _nvtx(name):
    """An NVTX range around a timed region (a profiler can select the timed
    launches by it); a no-op where NVTX is unavailable."""
    import contextlib
    try:
        import torch
        return torch.cuda.nvtx.range(name)
    except Exception:
        return contextlib.nullcontext()


def _time_plan(iqa, ctx, plan, stream, K, warmup, label=None):
    import contextlib
    import torch
    with torch.cuda.stream(stream):
        for _ in range(max(3, warmup)):
            iqa.iqa_plan_launch(plan, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream), (_nvtx(label) if label else contextlib.nullcontext()):
        e0.record(stream)
        for _ in range(K):
            iqa.iqa_plan_launch(plan, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    iqa.iqa_wait(ctx, stream, 60_000_000)
    return e0.elapsed_time(e1)


def _isolated(stream, fn, count, delay_cycles=200000):
    """Device times (us) of isolated launches: a GPU-side delay is queued
    ahead of each, so the launch is already queued when the events run; the
    first three are dropped."""
    import torch
    out = []
    for i in range(count):
        with torch.cuda.stream(stream):
            torch.cuda._sleep(delay_cycles)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fn(i)
            a1.record(stream)
        torch.cuda.synchronize()
        out.append(a0.elapsed_time(a1) * 1e3)
    return out[3:]


def _region_mean(stream, fn, K, delay_cycles=100000):
    """Mean device time (us) of an isolated launch from one event region:
    K (delay, launch) pairs minus K delays alone, which averages out the
    coarse tick of isolated event times."""
    import torch
    with torch.cuda.stream(stream):
        for i in range(3):
            torch.cuda._sleep(delay_cycles)
            fn(i)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        for i in range(K):
            torch.cuda._sleep(delay_cycles)
            fn(i)
        e[1].record(stream)
        e[2].record(stream)
        for i in range(K):
            torch.cuda._sleep(delay_cycles)
        e[3].record(stream)
    torch.cuda.synchronize()
    return (e[0].elapsed_time(e[1]) - e[2].elapsed_time(e[3])) * 1e3 / K


def small_pair_report(iqa, ctx, params, stream):
    """The small single pair (N=256, N_T=64, 16 tiles, FP32, 10 sources, seed
    0): one iqa_both call, isolated (median of 10, the paper's count, and the
    region mean) and back to back; its maps go to the CPU-baseline leg for
    the error against the oracle."""
    import torch
    from paper_2501_10653_gb300 import synth
    x, y = synth.small_pair()
    N, NT = 256, 64
    T = N // NT
    dev = torch.device("cuda", torch.cuda.current_device())
    # several copies, so that back-to-back launches rotate over distinct buffers
    C = 8
    dx = [torch.from_numpy(x).to(dev) for _ in range(C)]
    dy = [torch.from_numpy(y).to(dev) for _ in range(C)]
    lm = [torch.empty(T * T, device=dev) for _ in range(C)]
    am = [torch.empty(T * T, device=dev) for _ in range(C)]
    fn = lambda i: iqa.iqa_both(ctx, dx[i % C], dy[i % C], iqa.IQA_F32, N, NT, params,
                                lm[i % C], am[i % C], None, stream)
    iso = _isolated(stream, fn, 13)
    mean = _region_mean(stream, fn, 40)
    with torch.cuda.stream(stream):
        for i in range(10):
            fn(i)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(400):
            fn(i)
        e1.record(stream)
    torch.cuda.synchronize()
    b2b = e0.elapsed_time(e1) * 1e3 / 400

    # the same calls captured in a CUDA graph (no host launch cost), stream
    # ordered and as independent calls (each call's neighbours write other
    # maps, so the promise holds)
    def graph_us(independent):
        G = 8 * C
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INDEPENDENT_CALLS, independent)
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for i in range(G):
                    fn(i)
        finally:
            iqa.iqa_set_option(ctx, iqa.IQA_OPT_INDEPENDENT_CALLS, 0)
        with torch.cuda.stream(stream):
            g.replay()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(10):
                g.replay()
            g1.record(stream)
        torch.cuda.synchronize()
        return g0.elapsed_time(g1) * 1e3 / (10 * G)
    graph_b2b = graph_us(0)
    graph_indep = graph_us(1)
    return {"workload": "N=256 N_T=64 FP32 (16 tiles), 10 sources FWHM 3 px, flux 0.01..1, "
                        "noise sigma 1e-3, 3 faintest dropped, seed 0; one iqa_both call "
                        "per pair",
            "single_launch_us_median10": round(float(np.median(iso)), 3),
            "single_launch_us_mean": round(mean, 3),
            "back_to_back_us_per_pair": round(b2b, 3),
            "back_to_back_GBs": round(2 * N * N * 4 / (b2b * 1e-6) / 1e9, 1),
            "graph_back_to_back_us_per_pair": round(graph_b2b, 3),
            "graph_independent_calls_us_per_pair": round(graph_indep, 3),
            "launch": iqa.iqa_get_config(ctx, iqa.IQA_F32, N, NT, iqa.MAPS_BOTH).as_dict(),
            "_maps": (x, y, lm[0].cpu().numpy().astype(np.float64),
                      am[0].cpu().numpy().astype(np.float64))}


def precision_report(iqa, ctx, params, stream, batch=16, tune_iters=3):
    """The precision workload's size (N=8192, N_T=64, point + extended sources,
    1e4 dynamic range, sigma 5e-3) stored as FP32, FP16 and BF16: the batched
    throughput of each storage type, and pair 0's maps from those launches
    (returned apart: the per-tile errors against the FP64 oracle are formed
    in the CPU-baseline leg, ``precision_errors``)."""
    import torch
    from paper_2501_10653_gb300 import synth
    N, NT = 8192, 64
    T = N // NT
    x32, y32 = synth.precision_pair(0)
    out = {"workload": "N=8192 N_T=64, 33 sources (half extended, sigma 5-40 px), peak "
                       "flux 1e-4..1, noise sigma 5e-3, 10%% of sources dropped; %d copies of "
                       "the pair per launch" % batch}
    dev = torch.device("cuda", torch.cuda.current_device())
    maps_out = {}
    for name, code in (("f32", iqa.IQA_F32), ("f16", iqa.IQA_F16), ("bf16", iqa.IQA_BF16)):
        x, y = synth._cast(x32.astype(np.float64), name), synth._cast(y32.astype(np.float64), name)
        tx = torch.from_numpy(x.view(np.int16) if x.dtype == np.uint16 else x).to(dev)
        ty = torch.from_numpy(y.view(np.int16) if y.dtype == np.uint16 else y).to(dev)
        B = batch
        xs = [tx] + [tx.clone() for _ in range(B - 1)]
        ys = [ty] + [ty.clone() for _ in range(B - 1)]
        outs = [(torch.empty(T * T, device=dev), torch.empty(T * T, device=dev))
                for _ in range(B)]
        pairs = [iqa.make_pair(xs[i], ys[i], N, NT, *outs[i]) for i in range(B)]
        plan = iqa.iqa_plan_create(ctx, pairs, code, params, iqa.IQA_PLAN_GRAPH)
        if tune_iters > 0:
            out.setdefault("tuned", {})[name] = iqa.iqa_plan_autotune(plan, stream,
                                                                      tune_iters).as_dict()
        ms = _time_plan(iqa, ctx, plan, stream, 20, 3, label="precision_" + name)
        iqa.iqa_plan_destroy(plan)
        es = 4 if name == "f32" else 2
        out[name] = {
            "batched_GBs": round(20 * B * 2 * N * N * es / (ms * 1e-3) / 1e9, 1),
            "pixel_pairs_per_s": round(20 * B * N * N / (ms * 1e-3), 1),
        }
        # pair 0's maps, as the timed launches wrote them, for the error
        # figures of the CPU-baseline leg
        maps_out[name] = (x, y, outs[0][0].cpu().numpy(), outs[0][1].cpu().numpy())
        del xs, ys, outs, tx, ty
        torch.cuda.empty_cache()
    return out, (x32, y32, maps_out)


def merge_report(iqa, params, ctx, stream, x, y, K=200):
    """Eq. 3 / Eq. 4 merging (Section 3) from the exported per-tile sums of
    one N=2048, N_T=16 FP32 pair: merged maps at m = 2, 8 and the whole image
    (m = 128), each against computing the same coarser map from the pixels
    again (N_T' = m N_T); device time per call, back to back."""
    import torch
    N, NT = x.shape[0], 16
    T = N // NT
    sums = torch.empty((T * T, 4), dtype=torch.float64, device=x.device)
    lm = torch.empty(T * T, device=x.device)
    am = torch.empty(T * T, device=x.device)
    iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, NT, params, lm, am, sums, stream)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(5):
                fn()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(K):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / K

    out = {"workload": "one N=2048 FP32 pair, tile sums at N_T=16 (T=128)",
           "tile_map_us": round(timed(lambda: iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, NT,
                                                           params, lm, am, sums, stream)), 2)}
    for m in (2, 8, T):
        t = T // m
        ml = torch.empty(t * t, device=x.device)
        ma = torch.empty(t * t, device=x.device)
        rl = torch.empty(t * t, device=x.device)
        ra = torch.empty(t * t, device=x.device)
        merge_us = timed(lambda: iqa.iqa_merge(ctx, sums, T, m, params, ml, ma, None, stream))
        direct_us = timed(lambda: iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, NT * m, params, rl,
                                               ra, None, stream))
        out["m%d" % m] = {"merged_tiles": t * t, "merge_us": round(merge_us, 2),
                          "from_pixels_us": round(direct_us, 2),
                          "sums_bytes_read": T * T * 32}
    return out


SERVE_NS = (512, 1024, 2048, 4096, 8192, 16384)


def mixed_batch_report(iqa, ctx, params, stream, K=10):
    """The batched workload: 64 pairs, N from {1024, 2048, 4096, 8192}
    (weights 4:3:2:1), N_T from {32, 64, 128}, FP32; each pair a seeded sky of
    round(33 (N/2048)^2) Gaussian-beam sources (integer centres) over 2e-4
    noise, epoch 2 without the faintest 10% and with fresh noise, rendered on
    the device.  One persistent launch over all 64 (graph, autotuned) against
    one iqa_both launch per pair."""
    import math
    import torch
    from paper_2501_10653_gb300 import synth
    specs = synth.mixed_batch_specs()
    dev = torch.device("cuda", torch.cuda.current_device())
    xs, ys, outs, pairs = [], [], [], []
    total = 0
    for i, (N, NT) in enumerate(specs):
        cat = synth.serving_catalog(N, i, seed=2)
        cat2 = synth.catalog_without_faintest(cat, int(math.ceil(0.1 * len(cat["x"]))))
        x = torch.empty(N * N, device=dev)
        y = torch.empty(N * N, device=dev)
        iqa.iqa_render_epoch(ctx, cat, 2 * 10**6 + 2 * i, x, iqa.IQA_F32)
        iqa.iqa_render_epoch(ctx, cat2, 2 * 10**6 + 2 * i + 1, y, iqa.IQA_F32)
        T = N // NT
        o = (torch.empty(T * T, device=dev), torch.empty(T * T, device=dev))
        xs.append(x)
        ys.append(y)
        outs.append(o)
        pairs.append(iqa.make_pair(x, y, N, NT, *o))
        total += 2 * N * N * 4
    plan = iqa.iqa_plan_create(ctx, pairs, iqa.IQA_F32, params, iqa.IQA_PLAN_GRAPH)
    tuned = iqa.iqa_plan_autotune(plan, stream, 2).as_dict()
    ms = _time_plan(iqa, ctx, plan, stream, K, 2)
    iqa.iqa_plan_destroy(plan)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for (N, NT), x, y, o in zip(specs, xs, ys, outs):
            iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, NT, params, o[0], o[1], None, stream)
        e0.record(stream)
        for _ in range(K):
            for (N, NT), x, y, o in zip(specs, xs, ys, outs):
                iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, NT, params, o[0], o[1], None, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    per_pair_ms = e0.elapsed_time(e1)
    out = {"workload": "64 pairs, N in {1024,2048,4096,8192} (4:3:2:1), N_T in {32,64,128}, "
                       "FP32, skies rendered on the device", "input_bytes": total,
           "one_launch_us": round(ms * 1e3 / K, 1),
           "one_launch_GBs": round(K * total / (ms * 1e-3) / 1e9, 1),
           "one_launch_pairs_per_s": round(K * 64 / (ms * 1e-3), 1),
           "per_pair_launches_GBs": round(K * total / (per_pair_ms * 1e-3) / 1e9, 1),
           "per_pair_launches_pairs_per_s": round(K * 64 / (per_pair_ms * 1e-3), 1),
           "tuned": tuned}
    del xs, ys, outs
    torch.cuda.empty_cache()
    return out


def serving_report(iqa, ctx, seconds, rate=2000.0, n_refs=32, seed=4):
    """The serving workload: Poisson arrivals (rate per s, for `seconds`) of
    requests against n_refs resident reference skies (N uniform over
    512..16384, FP16), N_T uniform over {32, 64, 128}, each second epoch
    rendered on the device from its seed (2 sources dropped, a transient in
    half of them).  Served by the continuous-batching server, then by the
    one-pair-per-launch FP32 baseline on the same trace; plus a saturation
    burst for the maximum pairs/s of each."""
    from paper_2501_10653_gb300 import synth
    rng = np.random.default_rng([seed, 9])
    cats = {i: synth.serving_catalog(SERVE_NS[i % len(SERVE_NS)], i, seed=seed)
            for i in range(n_refs)}
    n = int(rate * seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    trace = []
    for i in range(n):
        rid = int(rng.integers(n_refs))
        cat = cats[rid]
        nsrc = len(cat["x"])
        drop = [int(v) for v in rng.choice(nsrc, size=min(2, nsrc), replace=False)]
        add = None
        if rng.random() < 0.5:
            N = cat["N"]
            add = (int(rng.integers(nsrc)), int(rng.integers(N)), int(rng.integers(N)),
                   float(np.exp(rng.uniform(np.log(0.01), 0.0))))
        trace.append(iqa.make_request(rid, int(rng.choice([32, 64, 128])), 10**9 + i,
                                      drop, add))

    def run(dtype, one_pair, timed, burst=None, marks=0):
        # steps of up to 32 pairs and 1 GB of input (a mean request is about
        # 239 MB in FP16): at saturation a step batches several requests
        srv = iqa.iqa_server_create(ctx, dtype=dtype, max_pairs_per_step=32,
                                    max_inflight_steps=4, pool_bytes=8 << 30,
                                    one_pair_per_launch=one_pair,
                                    max_step_bytes=1 << 30, params=PARAMS,
                                    time_kernels=marks)
        try:
            for rid, cat in cats.items():
                iqa.iqa_server_add_reference(srv, rid, cat, 7 + rid)
            reqs = trace if burst is None else trace[:burst]
            times = arrivals[:len(reqs)] if timed else np.zeros(len(reqs))
            t0 = time.perf_counter()
            iqa.iqa_server_run_trace(srv, reqs, times, timeout_s=600.0)
            wall = time.perf_counter() - t0
            st = iqa.iqa_server_get_stats(srv).as_dict()
            st["wall_s"] = round(wall, 3)
            return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()}
        finally:
            iqa.iqa_server_destroy(srv)

    burst = min(n, 2000)
    out = {
        "workload": "Poisson %.0f req/s for %.1f s (%d requests); %d resident FP16 reference "
                    "skies, N uniform over %s; N_T in {32,64,128}; epoch 2 rendered on the "
                    "device (2 sources dropped, a transient in half)" % (
                        rate, seconds, n, n_refs, list(SERVE_NS)),
        "served": run(iqa.IQA_F16, 0, True),
        "baseline_one_pair_per_launch_f32": run(iqa.IQA_F32, 1, True),
        "saturation_burst": burst,
        "served_saturation": run(iqa.IQA_F16, 0, False, burst),
        "baseline_saturation": run(iqa.IQA_F32, 1, False, burst),
    }
    # the same bursts again with timing marks around every step's two kernels
    # (the marks cut the launch overlap between them, so they stay out of the
    # runs above): device time per pair of the epoch generator and of the map
    # kernel, as they ran concurrently in up to four steps
    split = {}
    for name, dt, one in (("served", iqa.IQA_F16, 0), ("baseline", iqa.IQA_F32, 1)):
        r = run(dt, one, False, burst, marks=1)
        split[name] = {k: r[k] for k in ("pairs_per_s", "mean_pairs_per_step",
                                          "generator_ms_per_pair", "map_ms_per_pair",
                                          "mean_step_generator_ms", "mean_step_map_ms")}
    out["saturation_device_split"] = split
    return out


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
    from paper_2501_10653_gb300 import iqa

    N, NT = N_IMG, N_TILE
    T = N // NT
    B = max(1, args.batch)
    pair_bytes = 2 * N * N * 4
    ctx = iqa.iqa_create(local, 0)
    params = iqa.iqa_params(PARAMS["C1"], PARAMS["C2"], PARAMS["C"], PARAMS["D"])
    stream = torch.cuda.Stream(device=dev)

    # B distinct pairs per rank (independent replicas); one step = one
    # persistent launch over all B pairs
    host_pairs = _pool_pairs(rank, B)
    dx = [torch.from_numpy(x).to(dev) for x, _ in host_pairs]
    dy = [torch.from_numpy(y).to(dev) for _, y in host_pairs]
    lisi = [torch.empty(T * T, device=dev) for _ in range(B)]
    aug = [torch.empty(T * T, device=dev) for _ in range(B)]

    # Steps are direct launches of an independent plan (IQA_PLAN_INDEPENDENT):
    # back to back, each launch's CTAs are scheduled while the previous launch
    # drains (programmatic dependent launch) and copy their first units at
    # once; every other access waits for it.  A step writes only its own
    # maps, with the same values every time, so the plan's promise holds.
    # Stream-ordered launches of the same plan (no flag) and graph replays,
    # which cannot overlap across replays, are reported beside it.
    def make_plan(nt, flags=iqa.IQA_PLAN_INDEPENDENT):
        t = N // nt
        lm = lisi if nt == NT else [torch.empty(t * t, device=dev) for _ in range(B)]
        am = aug if nt == NT else [torch.empty(t * t, device=dev) for _ in range(B)]
        pairs = [iqa.make_pair(dx[i], dy[i], N, nt, lm[i], am[i]) for i in range(B)]
        return iqa.iqa_plan_create(ctx, pairs, iqa.IQA_F32, params, flags), (lm, am)

    plan, _ = make_plan(NT)
    tuned = (iqa.iqa_plan_autotune(plan, stream, args.tune_iters).as_dict()
             if args.tune_iters > 0 else None)
    info = iqa.iqa_plan_info(plan).as_dict()

    clocks = ClockSampler(local)
    clocks.start()
    K = max(1, args.steps)
    barrier(world)
    dev_ms = _time_plan(iqa, ctx, plan, stream, K, args.warmup, label="headline_timed")
    barrier(world)
    clk = clocks.stop()
    t_max_ms = max_over_ranks(dev_ms, world, dev)
    # end to end through the host-buffer entry point: one call per step over
    # the same B pairs in page-locked host memory, uploads pipelined with the
    # reductions, maps read back (measured right after the headline, before
    # the other reports fill host and device memory)
    hx = [torch.from_numpy(x).pin_memory() for x, _ in host_pairs]
    hy = [torch.from_numpy(y).pin_memory() for _, y in host_pairs]
    hl = [np.empty(T * T, np.float32) for _ in range(B)]
    ha = [np.empty(T * T, np.float32) for _ in range(B)]
    hpairs = [iqa.make_host_pair(hx[i], hy[i], N, NT, hl[i], ha[i]) for i in range(B)]
    iqa.iqa_both_host_many(ctx, hpairs, iqa.IQA_F32, params)
    # context for e2e: plain page-locked host -> device copies of the same
    # host buffers (one pair per repetition), before and after it
    scratch = torch.empty(N * N, device=dev)

    def plain_h2d():
        scratch.copy_(hx[0].view(-1), non_blocking=True)
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        for r in range(10):
            scratch.copy_(hx[r % B].view(-1), non_blocking=True)
            scratch.copy_(hy[r % B].view(-1), non_blocking=True)
        torch.cuda.synchronize()
        return 10 * pair_bytes / (time.perf_counter() - c0) / 1e9

    h2d_before = plain_h2d()
    # three blocks of E steps; the median block is reported (the host link is
    # shared with the machine's other GPUs, so one block can catch a transient)
    E = max(1, args.e2e_steps)
    blocks = []
    for _ in range(3):
        barrier(world)
        t0 = time.perf_counter()
        for i in range(E):
            iqa.iqa_both_host_many(ctx, hpairs, iqa.IQA_F32, params)
        blocks.append(max_over_ranks(time.perf_counter() - t0, world, dev))
    e2e_s = float(np.median(blocks))
    assert all(np.all(np.isfinite(v)) for v in hl + ha)
    h2d_gbs = max(h2d_before, plain_h2d())
    del scratch

    KG = max(10, min(K, 2000))
    other = {}
    for name, flags in (("stream_ordered", 0), ("graph", iqa.IQA_PLAN_GRAPH)):
        pl, _ = make_plan(NT, flags)
        if args.tune_iters > 0:
            iqa.iqa_plan_autotune(pl, stream, args.tune_iters)
        ms = _time_plan(iqa, ctx, pl, stream, KG, 3)
        iqa.iqa_plan_destroy(pl)
        other[name] = KG * B * pair_bytes / (ms * 1e-3) / 1e9
    graph_gbs = other["graph"]

    # one pair per launch (the plain call), back to back from a CUDA graph
    G = 4 * B
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        for i in range(B):
            iqa.iqa_both(ctx, dx[i], dy[i], iqa.IQA_F32, N, NT, params, lisi[i], aug[i],
                         None, stream)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        for i in range(G):
            j = i % B
            iqa.iqa_both(ctx, dx[j], dy[j], iqa.IQA_F32, N, NT, params, lisi[j], aug[j],
                         None, stream)
    reps = max(1, min(50, K // G + 1))
    with torch.cuda.stream(stream):
        g.replay()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(reps):
            g.replay()
        p1.record(stream)
    torch.cuda.synchronize()
    per_pair_us = p0.elapsed_time(p1) * 1e3 / (reps * G)
    # the same calls as independent calls (IQA_OPT_INDEPENDENT_CALLS: each one
    # loads and reduces its pixels while the call before it drains; every call
    # writes its own maps, so the promise holds), captured and replayed alike
    iqa.iqa_set_option(ctx, iqa.IQA_OPT_INDEPENDENT_CALLS, 1)
    try:
        gi = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gi, stream=stream):
            for i in range(G):
                j = i % B
                iqa.iqa_both(ctx, dx[j], dy[j], iqa.IQA_F32, N, NT, params, lisi[j], aug[j],
                             None, stream)
    finally:
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INDEPENDENT_CALLS, 0)
    with torch.cuda.stream(stream):
        gi.replay()
        p0.record(stream)
        for _ in range(reps):
            gi.replay()
        p1.record(stream)
    torch.cuda.synchronize()
    indep_call_us = p0.elapsed_time(p1) * 1e3 / (reps * G)
    del gi
    # one pair per launch through the plan API instead: B one-pair independent
    # plans launched directly back to back (each launch's first units stream
    # while the previous one drains)
    one_plans = [iqa.iqa_plan_create(ctx, [iqa.make_pair(dx[i], dy[i], N, NT, lisi[i], aug[i])],
                                     iqa.IQA_F32, params, iqa.IQA_PLAN_INDEPENDENT)
                 for i in range(B)]
    with torch.cuda.stream(stream):
        for i in range(3 * B):
            iqa.iqa_plan_launch(one_plans[i % B], stream)
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for i in range(reps * G):
            iqa.iqa_plan_launch(one_plans[i % B], stream)
        q1.record(stream)
    torch.cuda.synchronize()
    plan_pair_us = q0.elapsed_time(q1) * 1e3 / (reps * G)
    for p in one_plans:
        iqa.iqa_plan_destroy(p)
    def single_launches(fn, count):
        return _isolated(stream, lambda i: fn(i % B), count)

    both_j = lambda j: iqa.iqa_both(ctx, dx[j], dy[j], iqa.IQA_F32, N, NT, params, lisi[j],
                                    aug[j], None, stream)
    single = single_launches(both_j, 63)
    single_us = float(np.median(single))
    single_mean = _region_mean(stream, lambda i: both_j(i % B), 60)
    lisi_only = single_launches(lambda j: iqa.iqa_lisi(ctx, dx[j], dy[j], iqa.IQA_F32, N, NT,
                                                       params, lisi[j], None, stream), 13)
    aug_only = single_launches(lambda j: iqa.iqa_auglisi(ctx, dx[j], dy[j], iqa.IQA_F32, N, NT,
                                                         params, aug[j], None, stream), 13)
    plain_cfg = iqa.iqa_get_config(ctx, iqa.IQA_F32, N, NT, iqa.MAPS_BOTH).as_dict()
    # the floor of this way of timing: an empty kernel, isolated the same way
    floor = _isolated(stream, lambda i: torch.cuda._sleep(1), 23)
    floor_mean = _region_mean(stream, lambda i: torch.cuda._sleep(1), 60)
    # the paper's other timing form: one pair per call at every N_T of the sweep
    nt_single = {}
    for nt in PAPER_NT_SWEEP:
        t2 = N // nt
        lm2 = [torch.empty(t2 * t2, device=dev) for _ in range(2)]
        am2 = [torch.empty(t2 * t2, device=dev) for _ in range(2)]
        fn = (lambda nt_, lm_, am_: lambda i: iqa.iqa_both(
            ctx, dx[i % B], dy[i % B], iqa.IQA_F32, N, nt_, params, lm_[i % 2], am_[i % 2],
            None, stream))(nt, lm2, am2)
        iso = _isolated(stream, fn, 13)
        nt_single[str(nt)] = {"median10_us": round(float(np.median(iso)), 3),
                              "mean_us": round(_region_mean(stream, fn, 40), 3),
                              "launch": iqa.iqa_get_config(ctx, iqa.IQA_F32, N, nt,
                                                           iqa.MAPS_BOTH).as_dict()}
    small = small_pair_report(iqa, ctx, params, stream)

    # N_T sweep of the batched form (the paper's Fig. 1 axis)
    sweep = {}
    for nt in PAPER_NT_SWEEP:
        if nt == NT:
            sweep[str(nt)] = round(K * B * pair_bytes / (dev_ms * 1e-3) / 1e9, 1)
            continue
        pl, _keep = make_plan(nt)
        if args.tune_iters > 0:
            iqa.iqa_plan_autotune(pl, stream, args.tune_iters)
        ms = _time_plan(iqa, ctx, pl, stream, max(10, min(K, 200)), 3,
                        label="nt_sweep_%d" % nt)
        sweep[str(nt)] = round(max(10, min(K, 200)) * B * pair_bytes / (ms * 1e-3) / 1e9, 1)
        iqa.iqa_plan_destroy(pl)

    # the same step with the pairs stored in 16 bits (rounded to nearest):
    # half the bytes per pixel pair, so the rate in pixel pairs is the figure
    # to compare
    storage16 = {}
    for name, code, tdt in (("f16", iqa.IQA_F16, torch.float16),
                            ("bf16", iqa.IQA_BF16, torch.bfloat16)):
        hx16 = [t.to(tdt) for t in dx]
        hy16 = [t.to(tdt) for t in dy]
        pairs16 = [iqa.make_pair(hx16[i], hy16[i], N, NT, lisi[i], aug[i]) for i in range(B)]
        pl16 = iqa.iqa_plan_create(ctx, pairs16, code, params, iqa.IQA_PLAN_INDEPENDENT)
        tuned16 = (iqa.iqa_plan_autotune(pl16, stream, args.tune_iters).as_dict()
                   if args.tune_iters > 0 else None)
        K16 = max(10, min(K, 2000))
        ms = _time_plan(iqa, ctx, pl16, stream, K16, 3, label="storage_" + name)
        iqa.iqa_plan_destroy(pl16)
        # twice the pairs per launch (a second copy of each), so that a launch
        # moves the same bytes as the FP32 step: separates the per-launch cost
        # from the per-byte cost of the 16-bit kernel
        hx2 = hx16 + [t.clone() for t in hx16]
        hy2 = hy16 + [t.clone() for t in hy16]
        l2 = [torch.empty(T * T, device=dev) for _ in range(2 * B)]
        a2 = [torch.empty(T * T, device=dev) for _ in range(2 * B)]
        pl2 = iqa.iqa_plan_create(ctx, [iqa.make_pair(hx2[i], hy2[i], N, NT, l2[i], a2[i])
                                        for i in range(2 * B)], code, params,
                                  iqa.IQA_PLAN_INDEPENDENT)
        ms2 = _time_plan(iqa, ctx, pl2, stream, K16, 3)
        iqa.iqa_plan_destroy(pl2)
        storage16[name] = {
            "GBs": round(K16 * B * pair_bytes / 2 / (ms * 1e-3) / 1e9, 1),
            "pixel_pairs_per_s": round(K16 * B * N * N / (ms * 1e-3), 1),
            "us_per_pair": round(ms * 1e3 / (K16 * B), 3),
            "tuned": tuned16,
            "GBs_%d_pairs_per_launch" % (2 * B): round(K16 * 2 * B * pair_bytes / 2 /
                                                       (ms2 * 1e-3) / 1e9, 1)}
        del hx16, hy16, hx2, hy2, l2, a2

    prec, prec_maps = None, None
    if rank == 0 and world == 1 and not args.no_precision:
        prec, prec_maps = precision_report(iqa, ctx, params, stream, args.precision_batch,
                                           min(args.tune_iters, 3))

    # N sweep at N_T = 64 (the paper's other Fig. 1 axis), about the same bytes
    # per launch at every N, built on the device from the step's pairs:
    # N < 2048 as contiguous pieces of each 2048^2 image, N > 2048 as mosaics
    # of them; independent plans, autotuned like the rest
    nsweep = {}
    for n2 in PAPER_N_SWEEP:
        if n2 == N:
            continue
        if n2 < N:
            k = (N // n2) ** 2
            xs = [dx[i].reshape(-1)[j * n2 * n2:(j + 1) * n2 * n2]
                  for i in range(B) for j in range(k)]
            ys = [dy[i].reshape(-1)[j * n2 * n2:(j + 1) * n2 * n2]
                  for i in range(B) for j in range(k)]
        else:
            r = n2 // N

            def mosaic(imgs, c):
                t = [imgs[(c * r * r + q) % B].view(N, N) for q in range(r * r)]
                return torch.cat([torch.cat(t[a * r:(a + 1) * r], dim=1) for a in range(r)],
                                 dim=0).reshape(-1).contiguous()
            count = max(1, B // (r * r))
            xs = [mosaic(dx, c) for c in range(count)]
            ys = [mosaic(dy, c) for c in range(count)]
        t2 = n2 // NT
        outs = [(torch.empty(t2 * t2, device=dev), torch.empty(t2 * t2, device=dev))
                for _ in xs]
        pl = iqa.iqa_plan_create(ctx, [iqa.make_pair(xs[i], ys[i], n2, NT, *outs[i])
                                       for i in range(len(xs))],
                                 iqa.IQA_F32, params, iqa.IQA_PLAN_INDEPENDENT)
        if args.tune_iters > 0:
            iqa.iqa_plan_autotune(pl, stream, args.tune_iters)
        KS = max(10, min(K, 200))
        ms = _time_plan(iqa, ctx, pl, stream, KS, 3)
        iqa.iqa_plan_destroy(pl)
        nsweep[str(n2)] = {"pairs_per_launch": len(xs),
                           "us_per_pair": round(ms * 1e3 / (KS * len(xs)), 3),
                           "GBs": round(KS * len(xs) * 2 * n2 * n2 * 4 / (ms * 1e-3) / 1e9, 1)}
        del xs, ys, outs
    nsweep[str(N)] = {"pairs_per_launch": B, "us_per_pair": round(dev_ms * 1e3 / (K * B), 3),
                      "GBs": round(K * B * pair_bytes / (dev_ms * 1e-3) / 1e9, 1)}
    torch.cuda.empty_cache()

    merge = None
    if rank == 0 and world == 1 and not args.no_merge:
        merge = merge_report(iqa, params, ctx, stream, dx[0], dy[0])
    mixed = None
    if rank == 0 and world == 1 and not args.no_mixed:
        mixed = mixed_batch_report(iqa, ctx, params, stream)
    serve = None
    if rank == 0 and world == 1 and args.serve_seconds > 0:
        serve = serving_report(iqa, ctx, args.serve_seconds)

    total_bytes = sum_over_ranks(K * B * pair_bytes, world, dev)
    value = total_bytes / (t_max_ms * 1e-3) / 1e9
    peak, peak_src = measured_peak()
    per_launch_us = dev_ms * 1e3 / K
    achieved = B * pair_bytes / (per_launch_us * 1e-6) / 1e9
    e2e_bytes = sum_over_ranks(E * B * pair_bytes, world, dev)
    e2e_value = e2e_bytes / e2e_s / 1e9

    result = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(host_pairs[0][0], host_pairs[0][1], args.cpu_seconds)
            # error figures against the oracle (outside every timed region)
            small_pair_errors(small)
            if prec_maps is not None:
                precision_errors(prec_maps, prec)
        small.pop("_maps", None)
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s",
            "n_gpus": world, "steps": K, "warmup": max(3, args.warmup),
            "ms_per_step": round(t_max_ms / K, 6), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian-beam radio skies, no dataset)",
            "config": {"workload": WORKLOAD,
                       "N": N, "N_T": NT, "tiles_per_pair": T * T, "pairs_per_step": B,
                       "l2": "inputs larger than L2: each step reads %d MB of distinct "
                             "pairs" % (B * pair_bytes // 2 ** 20),
                       "params": PARAMS, "launch": info["config"], "tuned": tuned,
                       "timing": "CUDA events around K direct launches of an independent "
                                 "plan (IQA_PLAN_INDEPENDENT: each launch's first units "
                                 "stream while the previous launch drains); stream-ordered "
                                 "launches of the same plan in stream_ordered_GBs, graph "
                                 "replays in graph_replay_GBs, each autotuned alike",
                       "parallelism": "replicas x%d" % world},
            "pct_of_peak": round(100 * value / world / peak, 2),
            "stream_ordered_GBs": round(other["stream_ordered"], 1),
            "graph_replay_GBs": round(graph_gbs, 1),
            "pairs_per_s": round(value * 1e9 / pair_bytes, 1),
            "pixel_pairs_per_s": round(value * 1e9 / 8, 1),
            "us_per_pair": round(per_launch_us / B, 3),
            "one_pair_per_launch": {
                "GBs": round(pair_bytes / (per_pair_us * 1e-6) / 1e9, 1),
                "us_per_pair": round(per_pair_us, 3),
                "single_launch_us": round(single_us, 3),
                "single_launch_us_median10": round(float(np.median(single[:10])), 3),
                "single_launch_us_median60": round(single_us, 3),
                "single_launch_us_min": round(float(np.min(single)), 3),
                "single_launch_us_mean": round(float(np.mean(single)), 3),
                "single_launch_us_mean_of_60_in_one_region": round(single_mean, 3),
                "empty_kernel_single_launch_us_median": round(float(np.median(floor)), 3),
                "empty_kernel_single_launch_us_mean_of_60": round(floor_mean, 3),
                "nt_sweep_single_launch": nt_single,
                "lisi_only_single_us_median10": round(float(np.median(lisi_only)), 3),
                "auglisi_only_single_us_median10": round(float(np.median(aug_only)), 3),
                "launch": plain_cfg,
                "independent_calls_us_per_pair": round(indep_call_us, 3),
                "independent_calls_GBs": round(pair_bytes / (indep_call_us * 1e-6) / 1e9, 1),
                "independent_plans_us_per_pair": round(plan_pair_us, 3),
                "independent_plans_GBs": round(pair_bytes / (plan_pair_us * 1e-6) / 1e9, 1),
                "timing": "back-to-back iqa_both launches replayed from a CUDA graph; "
                          "single launches (60 of both maps, 10 of each map alone, 10 per "
                          "N_T) each with a GPU-side delay queued ahead, rotating over the "
                          "step's pairs so that no launch finds its pixels in L2; isolated "
                          "event times are quantised to about 2 us on this GPU, so the "
                          "region mean (60 delay+launch pairs in one event region, minus 60 "
                          "delays alone) is the finer figure; the empty kernel timed both "
                          "ways is the floor of the method (launch and event overhead)"},
            "small_pair_N256": small,
            "nt_sweep_GBs": sweep,
            "n_sweep_NT64": nsweep,
            "storage_16bit": storage16,
            "clocks": clk,
            "e2e": {"value": round(e2e_value, 2), "unit": "GB/s",
                    "h2d_bytes_per_step": B * pair_bytes,
                    "d2h_bytes_per_step": B * 2 * T * T * 4,
                    "ms_per_step": round(e2e_s * 1e3 / E, 4),
                    "api": "iqa_both_host_many over the step's %d pairs, page-locked "
                           "host buffers, uploads pipelined with reductions" % B,
                    "timing": "median of 3 blocks of %d steps" % E,
                    "blocks_GBs": [round(e2e_bytes / b / 1e9, 1) for b in blocks],
                    "plain_h2d_copy_GBs": round(h2d_gbs, 1)},
            "gpu_launches": K,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": profiled_traffic(B),
                         "algorithmic_bytes": B * pair_bytes,
                         "traffic_source": "ncu, %s%s" % (
                             PROFILED_TRAFFIC["capture"],
                             "" if B == PROFILED_TRAFFIC["pairs_per_launch"] else
                             ", scaled by pairs to %d" % B),
                         "peak_source": peak_src,
                         "kernel": "iqa_stream_kernel<float,%d,1,1> (persistent, TMA)"
                                   % info["config"]["threads"]},
            "cpu_baseline": cpu,
            "mixed_batch_64": mixed,
            "merge_eq3_eq4": merge,
            "precision_N8192": prec,
            "serving": serve,
            "paper_context": PAPER_H100,
        }
    iqa.iqa_plan_destroy(plan)
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
        "config": {"workload": WORKLOAD, "N": N, "N_T": NT, "params": PARAMS,
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
