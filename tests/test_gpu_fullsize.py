"""Parity at the workloads' full sizes, in the launch configurations that
bench.py times (needs a GPU):

* 32 distinct N=2048, N_T=64 FP32 pairs in one autotuned persistent launch
  of an independent plan, launched back to back: every tile against the
  oracle;
* the same 32 pairs at N_T = 16, 32, 128, 256, and stored in FP16 / BF16
  (the bench's N_T sweep and 16-bit steps): every tile of four pairs;
* the 64-pair mixed batch (N up to 8192, 7.9 GB) rendered on the device,
  one autotuned launch: sampled tiles;
* 16 pairs at N=8192, N_T=64 in FP16 and BF16, one launch: sampled tiles;
* served requests at N=8192 and 16384 (FP16): sampled tiles.

Sampled tiles are checked against the oracle on pixel windows that the host
mirror of the device generator (synth.render_epoch_window) makes, bit for
bit, so no oracle input comes from the CUDA path."""
import functools
import math

import numpy as np
import pytest

import parity
from paper_2501_10653_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}


@pytest.fixture(scope="module")
def ctx():
    from paper_2501_10653_gb300 import build, iqa
    build.build()
    h = iqa.iqa_create(0, 0)
    yield h
    iqa.iqa_destroy(h)


@functools.lru_cache(maxsize=None)
def _paper_pairs(dt, count=32):
    """The headline's seeded paper-scale pairs, stored as dt on the host."""
    return tuple(synth.paper_pair(pair_index=i, dtype=dt) for i in range(count))


def _picks(T, rng, k):
    return np.unique(np.concatenate([rng.integers(0, T * T, k),
                                     [0, T - 1, T * T - T, T * T - 1]]))


def _plan_run(ctx, pairs, code, tune_iters, launches, flags=None):
    import torch
    from paper_2501_10653_gb300 import iqa
    st = torch.cuda.Stream()
    flags = iqa.IQA_PLAN_GRAPH if flags is None else flags
    plan = iqa.iqa_plan_create(ctx, pairs, code, PARAMS, flags)
    try:
        if tune_iters:
            iqa.iqa_plan_autotune(plan, st, tune_iters)
        with torch.cuda.stream(st):
            for _ in range(launches):
                iqa.iqa_plan_launch(plan, st)
        torch.cuda.synchronize()
        iqa.iqa_wait(ctx, st, 30_000_000)
    finally:
        iqa.iqa_plan_destroy(plan)


def test_headline_configuration_every_tile(ctx, orc):
    """bench.py's timed step: 32 distinct paper-scale pairs (the same seeded
    inputs), one persistent launch of an independent plan, autotuned and
    launched directly back to back (each launch's head overlapping the
    previous one's tail)."""
    import torch
    from paper_2501_10653_gb300 import iqa
    N, NT, B = 2048, 64, 32
    T = N // NT
    host = [synth.paper_pair(pair_index=i) for i in range(B)]
    dev = [(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()) for x, y in host]
    outs = [(torch.full((T * T,), float("nan"), device="cuda"),
             torch.full((T * T,), float("nan"), device="cuda")) for _ in range(B)]
    pairs = [iqa.make_pair(d[0], d[1], N, NT, o[0], o[1]) for d, o in zip(dev, outs)]
    _plan_run(ctx, pairs, iqa.IQA_F32, 2, 5, iqa.IQA_PLAN_INDEPENDENT)
    for (x, y), (lm, am) in zip(host, outs):
        want = parity.oracle_maps(orc, x, y, NT, PARAMS)
        parity.assert_parity((lm.cpu().numpy(), am.cpu().numpy(), None), want, PARAMS)


@pytest.mark.parametrize("NT,dt", [(16, "f32"), (32, "f32"), (128, "f32"), (256, "f32"),
                                   (64, "f16"), (16, "f16"), (64, "bf16")])
def test_sweep_and_16bit_steps_full_size(ctx, orc, NT, dt):
    """bench.py's N_T sweep and 16-bit steps: the headline's 32 pairs at
    another N_T (units of several tile rows at N_T = 16 and 32), or rounded
    to 16 bits (units of 128K pixel pairs), one autotuned independent plan
    launched back to back; every tile of four of the pairs against the
    oracle on the stored pixels."""
    import torch
    from paper_2501_10653_gb300 import iqa
    N, B = 2048, 32
    T = N // NT
    code = {"f32": iqa.IQA_F32, "f16": iqa.IQA_F16, "bf16": iqa.IQA_BF16}[dt]
    # rounded to the storage type on the host (BF16 as bit patterns), so the
    # oracle reads the same stored pixels as the kernel
    host = _paper_pairs(dt, B)
    dev = [(parity.to_device(x), parity.to_device(y)) for x, y in host]
    outs = [(torch.full((T * T,), float("nan"), device="cuda"),
             torch.full((T * T,), float("nan"), device="cuda")) for _ in range(B)]
    pairs = [iqa.make_pair(d[0], d[1], N, NT, o[0], o[1]) for d, o in zip(dev, outs)]
    _plan_run(ctx, pairs, code, 2, 5, iqa.IQA_PLAN_INDEPENDENT)
    for i in (0, 13, 22, B - 1):
        x, y = host[i]
        want = parity.oracle_maps(orc, x, y, NT, PARAMS)
        lm, am = outs[i]
        parity.assert_parity((lm.cpu().numpy(), am.cpu().numpy(), None), want, PARAMS)
    del dev, outs
    torch.cuda.empty_cache()


def test_mixed_batch_full_size_sampled(ctx, orc):
    """bench.py's mixed batch: 64 pairs, N in {1024..8192}, N_T in {32,64,128},
    skies rendered on the device exactly as the bench renders them."""
    import torch
    from paper_2501_10653_gb300 import iqa
    specs = synth.mixed_batch_specs()
    xs, ys, outs, pairs, meta = [], [], [], [], []
    for i, (N, NT) in enumerate(specs):
        cat = synth.serving_catalog(N, i, seed=2)
        cat2 = synth.catalog_without_faintest(cat, int(math.ceil(0.1 * len(cat["x"]))))
        x = torch.empty(N * N, device="cuda")
        y = torch.empty(N * N, device="cuda")
        iqa.iqa_render_epoch(ctx, cat, 2 * 10**6 + 2 * i, x, iqa.IQA_F32)
        iqa.iqa_render_epoch(ctx, cat2, 2 * 10**6 + 2 * i + 1, y, iqa.IQA_F32)
        T = N // NT
        o = (torch.full((T * T,), float("nan"), device="cuda"),
             torch.full((T * T,), float("nan"), device="cuda"))
        xs.append(x)
        ys.append(y)
        outs.append(o)
        pairs.append(iqa.make_pair(x, y, N, NT, *o))
        meta.append((cat, cat2, 2 * 10**6 + 2 * i))
    _plan_run(ctx, pairs, iqa.IQA_F32, 2, 2)
    rng = np.random.default_rng(21)
    for i, ((N, NT), o, (cat, cat2, seed)) in enumerate(zip(specs, outs, meta)):
        T = N // NT
        picks = _picks(T, rng, 4)
        want = []
        for t in picks:
            r0, c0 = (t // T) * NT, (t % T) * NT
            xw = synth.render_epoch_window(cat, seed, r0, r0 + NT, c0, c0 + NT)
            yw = synth.render_epoch_window(cat2, seed + 1, r0, r0 + NT, c0, c0 + NT)
            want.append(parity.oracle_tile(orc, xw, yw, PARAMS))
        parity.assert_sampled(o[0].cpu().numpy(), o[1].cpu().numpy(), picks, want, PARAMS)
    del xs, ys, outs
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_precision_size_16bit_batch_sampled(ctx, orc, dt):
    """16 pairs at N=8192, N_T=64 stored in 16 bits, one persistent launch
    (the precision workload's size and launch), noise sigma 5e-3."""
    import torch
    from paper_2501_10653_gb300 import iqa
    N, NT, B = 8192, 64, 16
    T = N // NT
    code = {"f16": iqa.IQA_F16, "bf16": iqa.IQA_BF16}[dt]
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dt]
    cats, outs, pairs, keep = [], [], [], []
    for i in range(B):
        cat = synth.serving_catalog(N, i, seed=3, noise=5e-3)
        x = torch.empty(N * N, dtype=tdt, device="cuda")
        y = torch.empty(N * N, dtype=tdt, device="cuda")
        iqa.iqa_render_epoch(ctx, cat, 3 * 10**6 + 2 * i, x, code)
        iqa.iqa_render_epoch(ctx, cat, 3 * 10**6 + 2 * i + 1, y, code, drop=[0, 1])
        o = (torch.full((T * T,), float("nan"), device="cuda"),
             torch.full((T * T,), float("nan"), device="cuda"))
        cats.append(cat)
        outs.append(o)
        keep.append((x, y))
        pairs.append(iqa.make_pair(x, y, N, NT, *o))
    _plan_run(ctx, pairs, code, 0, 2)
    rng = np.random.default_rng(33)
    for i, (cat, o) in enumerate(zip(cats, outs)):
        picks = _picks(T, rng, 6)
        want = []
        for t in picks:
            r0, c0 = (t // T) * NT, (t % T) * NT
            xw = synth.render_epoch_window(cat, 3 * 10**6 + 2 * i, r0, r0 + NT, c0, c0 + NT,
                                           dtype=dt)
            yw = synth.render_epoch_window(cat, 3 * 10**6 + 2 * i + 1, r0, r0 + NT, c0,
                                           c0 + NT, drop=[0, 1], dtype=dt)
            want.append(parity.oracle_tile(orc, xw, yw, PARAMS))
        parity.assert_sampled(o[0].cpu().numpy(), o[1].cpu().numpy(), picks, want, PARAMS)
    del keep, outs
    torch.cuda.empty_cache()


def test_served_requests_at_full_size_sampled(ctx, orc):
    """The serving workload's largest sizes (N = 8192 and 16384, FP16), with
    drops and transients, served in batched steps."""
    import time
    from paper_2501_10653_gb300 import iqa
    srv = iqa.iqa_server_create(ctx, dtype=iqa.IQA_F16, max_pairs_per_step=8,
                                max_inflight_steps=2, pool_bytes=4 << 30, params=PARAMS)
    try:
        cats = {}
        for rid, N in ((0, 8192), (1, 16384)):
            cats[rid] = synth.serving_catalog(N, rid)
            iqa.iqa_server_add_reference(srv, rid, cats[rid], 900 + rid)
        reqs = [(0, 64, 41, [0, 3], (2, 4000, 5000, 0.4)), (1, 128, 42, [1], None),
                (1, 32, 43, [], (5, 16000, 300, 1.2)), (0, 32, 44, [2], None)]
        hs = [iqa.iqa_submit(srv, iqa.make_request(r, nt, sd, dr, ad))
              for r, nt, sd, dr, ad in reqs]
        t0 = time.time()
        for h in hs:
            while iqa.iqa_poll(srv, h, 200_000) == iqa.IQA_PENDING:
                assert time.time() - t0 < 120
        rng = np.random.default_rng(44)
        for h, (rid, NT, seed, drop, add) in zip(hs, reqs):
            assert iqa.iqa_poll(srv, h, 0) == iqa.IQA_OK
            cat = cats[rid]
            N = cat["N"]
            T = N // NT
            lm = np.full(T * T, np.nan, np.float32)
            am = np.full(T * T, np.nan, np.float32)
            iqa.iqa_result(srv, h, lm, am)
            picks = _picks(T, rng, 6)
            if add is not None:  # the tile holding the transient's centre
                picks = np.unique(np.append(picks, (add[2] // NT) * T + add[1] // NT))
            want = []
            for t in picks:
                r0, c0 = (t // T) * NT, (t % T) * NT
                xw = synth.render_epoch_window(cat, 900 + rid, r0, r0 + NT, c0, c0 + NT,
                                               dtype="f16")
                yw = synth.render_epoch_window(cat, seed, r0, r0 + NT, c0, c0 + NT, drop=drop,
                                               add=add, dtype="f16")
                want.append(parity.oracle_tile(orc, xw, yw, PARAMS))
            parity.assert_sampled(lm, am, picks, want, PARAMS)
    finally:
        iqa.iqa_server_destroy(srv)


def test_largest_image_both_kernels_sampled(ctx, orc):
    """N = 32768 FP32 (8 GB per pair, 2^30 pixels per image, 262144 tiles at
    N_T = 64): the one-pair kernel and a one-pair persistent plan agree bit for
    bit on every tile, and sampled tiles match the oracle; N_T = N (one tile of
    the whole image, split over a cluster) matches it too."""
    import torch
    from paper_2501_10653_gb300 import iqa
    N, NT = 32768, 64
    T = N // NT
    cat = synth.serving_catalog(N, 7, seed=5)
    x = torch.empty(N * N, device="cuda")
    y = torch.empty(N * N, device="cuda")
    iqa.iqa_render_epoch(ctx, cat, 5001, x, iqa.IQA_F32)
    iqa.iqa_render_epoch(ctx, cat, 5002, y, iqa.IQA_F32, drop=[0, 1, 2], add=(3, 20000, 777, 0.9))
    st = torch.cuda.current_stream()
    l1 = torch.full((T * T,), float("nan"), device="cuda")
    a1 = torch.full((T * T,), float("nan"), device="cuda")
    iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, NT, PARAMS, l1, a1, None, st)
    l2 = torch.full((T * T,), float("nan"), device="cuda")
    a2 = torch.full((T * T,), float("nan"), device="cuda")
    _plan_run(ctx, [iqa.make_pair(x, y, N, NT, l2, a2)], iqa.IQA_F32, 0, 1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(55)
    picks = np.unique(np.append(_picks(T, rng, 12), (777 // NT) * T + 20000 // NT))
    want = []
    for t in picks:
        r0, c0 = (t // T) * NT, (t % T) * NT
        xw = synth.render_epoch_window(cat, 5001, r0, r0 + NT, c0, c0 + NT)
        yw = synth.render_epoch_window(cat, 5002, r0, r0 + NT, c0, c0 + NT, drop=[0, 1, 2],
                                       add=(3, 20000, 777, 0.9))
        want.append(parity.oracle_tile(orc, xw, yw, PARAMS))
    for lm, am in ((l1, a1), (l2, a2)):
        parity.assert_sampled(lm.cpu().numpy(), am.cpu().numpy(), picks, want, PARAMS)
    # the two kernels sum in different orders: equal within the parity bound
    parity.assert_lisi_close(l2.cpu().numpy(), l1.cpu().numpy().astype(np.float64))
    # one tile of the whole image: the sums against the sums of all 64-tiles
    s_all = torch.empty((T * T, 4), dtype=torch.float64, device="cuda")
    iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, NT, PARAMS, l1, a1, s_all, st)
    s_one = torch.empty((1, 4), dtype=torch.float64, device="cuda")
    lw = torch.empty(1, device="cuda")
    aw = torch.empty(1, device="cuda")
    iqa.iqa_both(ctx, x, y, iqa.IQA_F32, N, N, PARAMS, lw, aw, s_one, st)
    torch.cuda.synchronize()
    tot = s_all.cpu().numpy().sum(axis=0)
    one = s_one.cpu().numpy()[0]
    assert np.all(np.abs(one - tot) <= 1e-5 * np.abs(tot))
    del x, y, l1, a1, l2, a2, s_all
    torch.cuda.empty_cache()
