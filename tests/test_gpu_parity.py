"""CUDA path against the FP64 oracle, through the C-ABI (needs a GPU).

Inputs are the seeded synthetic skies of ``paper_2501_10653_gb300.synth``;
every comparison is element by element on all tiles (or, at full size, on
sampled tiles the oracle computes one by one), with the tolerance stated in
``tests/parity.py``.
"""
import itertools

import numpy as np
import pytest

import parity
from paper_2501_10653_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_10653_gb300 import build, iqa
    build.build()
    assert torch.cuda.is_available()
    h = iqa.iqa_create(0, 0)
    yield h
    iqa.iqa_destroy(h)


@pytest.fixture(scope="module")
def small():
    return synth.small_pair()


@pytest.fixture(scope="module")
def paper():
    return synth.paper_pair()


def test_small_pair_all_outputs(ctx, orc, small):
    x, y = small
    want = parity.oracle_maps(orc, x, y, 64, PARAMS)
    for which in ("both", "lisi", "aug", "both_nosums"):
        got = parity.gpu_maps(ctx, x, y, 64, PARAMS, which)
        parity.assert_parity(got, want, PARAMS)


@pytest.mark.parametrize("NT", synth.PAPER_NT_SWEEP)
def test_paper_pair_nt_sweep(ctx, orc, paper, NT):
    x, y = paper
    want = parity.oracle_maps(orc, x, y, NT, PARAMS)
    got = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    parity.assert_parity(got, want, PARAMS)


def _all_configs(N, NT):
    T = N // NT
    for threads, ilp, vector in itertools.product((128, 256, 512), (2, 4, 8), (1, 0)):
        if vector == 0 and (threads, ilp) != (256, 8):
            continue
        for TX in [d for d in range(1, min(T, 64) + 1) if T % d == 0]:
            for S in [s for s in range(1, 9) if NT % s == 0]:
                yield dict(threads=threads, ilp=ilp, tiles_across=TX, split=S,
                           vector=vector, variant=0)


@pytest.mark.parametrize("N,NT", [(512, 16), (512, 64), (512, 256), (480, 48),
                                  (384, 128), (512, 512)])
def test_every_launch_shape(ctx, orc, N, NT):
    """Every valid launch shape gives oracle parity (several tiles per unit,
    clusters of 2..8 CTAs per tile, ragged per-thread item counts)."""
    from paper_2501_10653_gb300 import iqa
    x, y = synth.paper_pair(N=N)
    want = parity.oracle_maps(orc, x, y, NT, PARAMS)
    dx, dy = parity.to_device(x), parity.to_device(y)
    n_ok = 0
    for cfg in _all_configs(N, NT):
        try:
            iqa.iqa_set_config(ctx, iqa.IQA_F32, N, NT, iqa.MAPS_BOTH, cfg)
        except iqa.IqaError as e:
            assert e.status == iqa.IQA_ERR_INVALID_ARG
            continue
        got = parity.gpu_maps(ctx, x, y, NT, PARAMS, dx=dx, dy=dy)
        parity.assert_parity(got, want, PARAMS)
        n_ok += 1
    iqa.iqa_set_config(ctx, iqa.IQA_F32, N, NT, iqa.MAPS_BOTH, None)
    assert n_ok >= 3


@pytest.mark.parametrize("N,NT", [(100, 10), (96, 12), (200, 40), (66, 33), (8, 8)])
def test_odd_shapes_scalar_and_vector(ctx, orc, N, NT):
    """Tiles that are not whole 16-byte vectors take the scalar path."""
    x, y = synth.paper_pair(N=N)
    want = parity.oracle_maps(orc, x, y, NT, PARAMS)
    parity.assert_parity(parity.gpu_maps(ctx, x, y, NT, PARAMS), want, PARAMS)


def test_misaligned_pointers_use_scalar_path(ctx, orc):
    import torch
    N, NT = 256, 32
    x, y = synth.paper_pair(N=N)
    want = parity.oracle_maps(orc, x, y, NT, PARAMS)
    bx = torch.zeros(N * N + 1, dtype=torch.float32, device="cuda")
    by = torch.zeros(N * N + 3, dtype=torch.float32, device="cuda")
    bx[1:].copy_(torch.from_numpy(x.ravel()))
    by[3:].copy_(torch.from_numpy(y.ravel()))
    got = parity.gpu_maps(ctx, x, y, NT, PARAMS, dx=bx[1:], dy=by[3:])
    parity.assert_parity(got, want, PARAMS)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
@pytest.mark.parametrize("NT", [16, 64, 256])
def test_16bit_storage_against_oracle_on_rounded_inputs(ctx, orc, dt, NT):
    x, y = synth.paper_pair(N=1024, dtype=dt)
    want = parity.oracle_maps(orc, x, y, NT, PARAMS)
    parity.assert_parity(parity.gpu_maps(ctx, x, y, NT, PARAMS), want, PARAMS)


def test_other_constants(ctx, orc, paper):
    x, y = paper
    p = {"C1": 1e-3, "C2": 0.5, "C": 0.25, "D": 0.125}
    want = parity.oracle_maps(orc, x, y, 64, p)
    parity.assert_parity(parity.gpu_maps(ctx, x, y, 64, p), want, p)


def test_all_zero_and_negative_tiles_exact(ctx):
    """Clamped-to-zero tiles: LISI exactly 0, augLISI exactly 1."""
    N = 256
    x = -np.abs(np.random.default_rng(1).standard_normal((N, N))).astype(np.float32)
    y = np.zeros((N, N), np.float32)
    y[::3, ::5] = np.nan
    l, a, s = parity.gpu_maps(ctx, x, y, 32, PARAMS)
    assert np.all(l == 0.0) and np.all(a == 1.0) and np.all(s == 0.0)


def test_identical_inputs(ctx, orc, paper):
    """x = y: augLISI exactly 1, LISI = Sx/(Sx + C2) within tolerance."""
    x, _ = paper
    l, a, s = parity.gpu_maps(ctx, x, x, 64, PARAMS)
    assert np.all(a == 1.0)
    _, _, osum = parity.oracle_maps(orc, x, x, 64, PARAMS)
    sx = osum[:, 2]
    parity.assert_lisi_close(l, sx / (sx + PARAMS["C2"]))


def test_nan_pixels_read_as_zero(ctx, orc, paper):
    x, y = paper
    x = x.copy()
    y = y.copy()
    rng = np.random.default_rng(5)
    x[rng.random(x.shape) < 0.01] = np.nan
    y[rng.random(y.shape) < 0.01] = np.nan
    want = parity.oracle_maps(orc, x, y, 64, PARAMS)
    parity.assert_parity(parity.gpu_maps(ctx, x, y, 64, PARAMS), want, PARAMS)


def test_tile_markers_bit_exact_indexing(ctx):
    """Changing one tile of y changes exactly its own entry of each map."""
    import torch
    from paper_2501_10653_gb300 import iqa
    N, NT = 512, 64
    T = N // NT
    x, y = synth.paper_pair(N=N)
    base_l, base_a, _ = parity.gpu_maps(ctx, x, y, NT, PARAMS, "both_nosums")
    for r in range(T):
        for c in range(T):
            y2 = y.copy()
            y2[r * NT + 5, c * NT + 7] += 0.5
            l, a, _ = parity.gpu_maps(ctx, x, y2, NT, PARAMS, "both_nosums")
            dl = np.argwhere(l.ravel() != base_l.ravel()).ravel().tolist()
            da = np.argwhere(a.ravel() != base_a.ravel()).ravel().tolist()
            assert dl == [r * T + c] and da == [r * T + c], (r, c, dl, da)


def test_inputs_not_written_and_deterministic(ctx, paper):
    import torch
    x, y = paper
    dx, dy = parity.to_device(x), parity.to_device(y)
    r1 = parity.gpu_maps(ctx, x, y, 64, PARAMS, dx=dx, dy=dy)
    r2 = parity.gpu_maps(ctx, x, y, 64, PARAMS, dx=dx, dy=dy)
    for u, v in zip(r1, r2):
        assert np.array_equal(u, v)
    assert np.array_equal(dx.cpu().numpy(), x)
    assert np.array_equal(dy.cpu().numpy(), y)


def test_host_path_matches_device_path_bitwise(ctx, paper):
    from paper_2501_10653_gb300 import iqa
    import torch
    x, y = paper
    N, NT = 2048, 64
    T = N // NT
    dev = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    hx = torch.from_numpy(x).pin_memory()
    hy = torch.from_numpy(y).pin_memory()
    l = np.full((T, T), np.nan, np.float32)
    a = np.full((T, T), np.nan, np.float32)
    s = np.full((T * T, 4), np.nan, np.float64)
    iqa.iqa_both_host(ctx, hx, hy, iqa.IQA_F32, N, NT, PARAMS, l, a, s)
    assert np.array_equal(l, dev[0]) and np.array_equal(a, dev[1])
    assert np.array_equal(s, dev[2])
    # pageable host memory works too
    l2 = np.zeros_like(l)
    iqa.iqa_both_host(ctx, x, y, iqa.IQA_F32, N, NT, PARAMS, l2, None, None)
    assert np.array_equal(l2, dev[0])


def test_full_size_sampled_tiles(ctx, orc):
    """N = 8192, N_T = 64 (the precision workload's size), FP32: sampled tiles
    against the oracle computed tile by tile."""
    x, y = synth.precision_pair(0)
    N, NT = 8192, 64
    T = N // NT
    got = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    rng = np.random.default_rng(9)
    pick = np.unique(np.concatenate([rng.integers(0, T * T, 200),
                                     [0, T - 1, T * T - T, T * T - 1]]))
    osums = orc.tile_sums(x, y, NT, PARAMS["C1"], tiles=pick)
    A, B, Sx, Sy = osums.T
    D = PARAMS["C1"] / 2
    ol = D * A / (np.maximum(Sx, Sy) + PARAMS["C2"])
    oa = 1 - B / (Sx + Sy + PARAMS["C"])
    r = B / (Sx + Sy + PARAMS["C"])
    parity.assert_lisi_close(got[0].ravel()[pick], ol)
    parity.assert_aug_close(got[1].ravel()[pick], oa, r)
    parity.assert_sums_close(got[2][pick], osums)


def test_whole_image_as_one_tile(ctx, orc, paper):
    """N_T = N: one tile over the whole 2048^2 image (a cluster of CTAs)."""
    x, y = paper
    want = parity.oracle_maps(orc, x, y, 2048, PARAMS)
    parity.assert_parity(parity.gpu_maps(ctx, x, y, 2048, PARAMS), want, PARAMS)


def test_bad_arguments_rejected(ctx):
    import torch
    from paper_2501_10653_gb300 import iqa
    d = torch.zeros(64 * 64, device="cuda")
    m = torch.zeros(16, device="cuda")
    cases = [
        dict(x=None, y=d, N=64, NT=16, m=m),
        dict(x=d, y=d, N=64, NT=12, m=m),
        dict(x=d, y=d, N=0, NT=16, m=m),
        dict(x=d, y=d, N=64, NT=0, m=m),
        dict(x=d, y=d, N=64, NT=128, m=m),
    ]
    for c in cases:
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_both(ctx, c["x"], c["y"], iqa.IQA_F32, c["N"], c["NT"], None,
                         c["m"], None)
        assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_both(ctx, d, d, iqa.IQA_F32, 64, 16, {"C1": 0.0}, m, None)
    assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_both(ctx, d, d, 7, 64, 16, None, m, None)
    assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_both(ctx, d, d, iqa.IQA_F32, 64, 16, None, None, None)
    assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
    torch.cuda.synchronize()


def _stream_configs(N, NT, es):
    V = 16 // es
    T = N // NT
    for threads in (128, 256, 512):
        for TX in [d for d in range(1, 65) if T % d == 0 and (d * NT <= 256 or (
                d * NT <= 1024 and d * NT % 256 == 0 and N % 256 == 0))]:
            for stage_kb in (2, 4, 8, 16):
                for stages, cps in ((4, 1), (8, 1), (3, 2)):
                    yield dict(variant=1, threads=threads, tiles_across=TX,
                               stages=stages, stage_kb=stage_kb, ctas_per_sm=cps)


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("N,NT", [(512, 16), (512, 64), (512, 256), (480, 48), (384, 128)])
def test_tma_persistent_kernel_every_shape(ctx, orc, dt, N, NT):
    """The persistent TMA-pipelined kernel (variant 1) against the oracle over
    every valid launch shape: consumer counts, units of several tiles (up to
    1024 elements wide, copied as 3-D boxes of 256-element segments), stage
    sizes that split a tile into 1..64 chunks, ring depths, 1 or 2 CTAs/SM."""
    from paper_2501_10653_gb300 import iqa
    es = 4 if dt == "f32" else 2
    if NT % (16 // es):
        pytest.skip("tile not a whole number of 16-byte vectors")
    x, y = synth.paper_pair(N=N, dtype=dt)
    want = parity.oracle_maps(orc, x, y, NT, PARAMS)
    dx, dy = parity.to_device(x), parity.to_device(y)
    code = parity.dtype_code(x)
    n_ok = 0
    for cfg in _stream_configs(N, NT, es):
        try:
            iqa.iqa_set_config(ctx, code, N, NT, iqa.MAPS_BOTH, cfg)
        except iqa.IqaError as e:
            assert e.status == iqa.IQA_ERR_INVALID_ARG
            continue
        got = parity.gpu_maps(ctx, x, y, NT, PARAMS, dx=dx, dy=dy)
        iqa.iqa_wait(ctx, None, 10_000_000)
        parity.assert_parity(got, want, PARAMS)
        n_ok += 1
    iqa.iqa_set_config(ctx, code, N, NT, iqa.MAPS_BOTH, None)
    assert n_ok >= 3


@pytest.mark.parametrize("which", ["lisi", "aug", "both_nosums"])
def test_tma_kernel_single_maps(ctx, orc, paper, which):
    from paper_2501_10653_gb300 import iqa
    x, y = paper
    maps = {"lisi": iqa.MAPS_LISI, "aug": iqa.MAPS_AUGLISI, "both_nosums": iqa.MAPS_BOTH}[which]
    iqa.iqa_set_config(ctx, iqa.IQA_F32, 2048, 64, maps,
                       dict(variant=1, threads=256, tiles_across=1, stages=8, stage_kb=8))
    want = parity.oracle_maps(orc, x, y, 64, PARAMS)
    got = parity.gpu_maps(ctx, x, y, 64, PARAMS, which)
    iqa.iqa_set_config(ctx, iqa.IQA_F32, 2048, 64, maps, None)
    parity.assert_parity(got, want, PARAMS)


# m^2 <= 16: a thread per merged tile; <= 8192: a warp; larger (whole image at
# N_T = 16: 16384 tiles; 4 blocks of 4096 at m = 64 use warps): an 8-CTA cluster
@pytest.mark.parametrize("NT,m", [(16, 2), (16, 8), (32, 4), (64, 32), (64, 1), (128, 16),
                                  (16, 64), (16, 128), (8, 256), (8, 128)])
def test_merge_eq3_eq4_against_oracle(ctx, orc, paper, NT, m):
    """Eq. 3 / Eq. 4 merging of m x m tile blocks (m = T: the whole image) from
    the GPU's per-tile sums, against the oracle's merge (Eq. 3 / Eq. 4 in the
    paper's form) and against the oracle computed directly at N_T' = m N_T."""
    import torch
    import oracle
    from paper_2501_10653_gb300 import iqa
    x, y = paper
    N = 2048
    T = N // NT
    M = T // m
    _, _, sums = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    ds = torch.from_numpy(sums).cuda()
    ml = torch.full((M * M,), float("nan"), device="cuda")
    ma = torch.full((M * M,), float("nan"), device="cuda")
    msum = torch.full((M * M, 4), float("nan"), device="cuda", dtype=torch.float64)
    iqa.iqa_merge(ctx, ds, T, m, PARAMS, ml, ma, msum, torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = (ml.cpu().numpy(), ma.cpu().numpy(), msum.cpu().numpy())
    direct = parity.oracle_maps(orc, x, y, NT * m, PARAMS)
    parity.assert_parity(got, direct, PARAMS)
    ol, oa, osums = parity.oracle_maps(orc, x, y, NT, PARAMS)
    el, ea = oracle.merge_tiles(ol, oa, osums, m, PARAMS["C2"], PARAMS["C"])
    r = direct[2][:, 1] / (direct[2][:, 2] + direct[2][:, 3] + PARAMS["C"])
    parity.assert_lisi_close(got[0], el.ravel())
    parity.assert_aug_close(got[1], ea.ravel(), r)


def test_merge_repeats_bit_for_bit(ctx, paper):
    """Every merge shape sums in an order fixed by the launch: repeated calls
    agree bit for bit."""
    import torch
    from paper_2501_10653_gb300 import iqa
    x, y = paper
    NT = 8
    T = 2048 // NT
    _, _, sums = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    ds = torch.from_numpy(sums).cuda()
    for m in (2, 16, 256):
        M = T // m
        outs = []
        for _ in range(3):
            ms = torch.empty((M * M, 4), device="cuda", dtype=torch.float64)
            iqa.iqa_merge(ctx, ds, T, m, PARAMS, None, None, ms, torch.cuda.current_stream())
            torch.cuda.synchronize()
            outs.append(ms.cpu().numpy())
        assert all(np.array_equal(outs[0].view(np.uint64), o.view(np.uint64)) for o in outs)


def test_merge_rejects_bad_factor(ctx):
    import torch
    from paper_2501_10653_gb300 import iqa
    s = torch.zeros((64, 4), device="cuda", dtype=torch.float64)
    o = torch.zeros(64, device="cuda")
    for T, m in ((8, 3), (8, 0), (8, 16)):
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_merge(ctx, s, T, m, PARAMS, o, None)
        assert ei.value.status == iqa.IQA_ERR_INVALID_ARG


def test_host_many_pipelined_matches_device_path(ctx, orc):
    """iqa_both_host_many over mixed pairs (two device slots, uploads overlapped
    with reductions) gives the device path's bits for every pair."""
    import torch
    from paper_2501_10653_gb300 import iqa
    specs = [(512, 64), (1024, 32), (256, 16), (512, 128), (1024, 64)]
    pairs, outs, hosts = [], [], []
    for i, (N, NT) in enumerate(specs):
        x, y = synth.mixed_batch_pair(i, N, seed=7)
        hx = torch.from_numpy(x).pin_memory()
        hy = torch.from_numpy(y).pin_memory()
        T = N // NT
        o = (np.full(T * T, np.nan, np.float32), np.full(T * T, np.nan, np.float32),
             np.full((T * T, 4), np.nan))
        hosts.append((x, y, hx, hy))
        outs.append(o)
        pairs.append(iqa.make_host_pair(hx, hy, N, NT, *o))
    iqa.iqa_both_host_many(ctx, pairs, iqa.IQA_F32, PARAMS)
    for (N, NT), (x, y, _, _), o in zip(specs, hosts, outs):
        dev = parity.gpu_maps(ctx, x, y, NT, PARAMS)
        assert np.array_equal(o[0], dev[0].ravel()) and np.array_equal(o[1], dev[1].ravel())
        assert np.array_equal(o[2], dev[2])
        parity.assert_parity(dev, parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_full_size_16bit_sampled_tiles(ctx, orc, dt):
    """N = 8192, N_T = 64 with 16-bit storage (the precision workload's size):
    sampled tiles against the oracle on the rounded inputs (the accumulation
    bound, 1e-5 relative)."""
    x, y = synth.precision_pair(0, dtype=dt)
    N, NT = 8192, 64
    T = N // NT
    got = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    rng = np.random.default_rng(10)
    pick = np.unique(np.concatenate([rng.integers(0, T * T, 150), [0, T * T - 1]]))
    osums = orc.tile_sums(parity.widen(x), parity.widen(y), NT, PARAMS["C1"], tiles=pick)
    A, B, Sx, Sy = osums.T
    D = PARAMS["C1"] / 2
    r = B / (Sx + Sy + PARAMS["C"])
    parity.assert_lisi_close(got[0].ravel()[pick], D * A / (np.maximum(Sx, Sy) + PARAMS["C2"]))
    parity.assert_aug_close(got[1].ravel()[pick], 1 - r, r)
    parity.assert_sums_close(got[2][pick], osums)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_16bit_nan_and_negative_pixels_read_as_zero(ctx, orc, dt):
    """16-bit pixels are clamped in packed form: NaN and negatives read as 0."""
    x, y = synth.paper_pair(N=512, dtype=dt)
    x = x.copy()
    y = y.copy()
    rng = np.random.default_rng(6)
    nan_bits = np.uint16(0x7E00) if dt == "f16" else np.uint16(0x7FC0)
    for a in (x, y):
        v = a.view(np.uint16)
        v[rng.random(v.shape) < 0.02] = nan_bits
    want = parity.oracle_maps(orc, x, y, 64, PARAMS)
    parity.assert_parity(parity.gpu_maps(ctx, x, y, 64, PARAMS), want, PARAMS)


def _cancelling_pair(dt):
    """y = 0 and x constant a_t = 1 + k_t / 64 per 16x16 tile, k_t in -3..3:
    r = B / (Sx + C) = a_t^2 m / (a_t m + C) is within 1/16 of 1, so
    aug = 1 - r cancels (aug = C / (m + C), about 4e-9, at k_t = 0).  Every
    term and every partial sum is a multiple of 2^-12 below 2^9, so the GPU's
    FP32 sums are exact and aug's accuracy is the combine's alone."""
    N, NT = 128, 16
    T = N // NT
    k = (np.arange(T * T) % 7 - 3).reshape(T, T)
    a = (1.0 + k / 64.0).astype(np.float32)
    x = np.kron(a, np.ones((NT, NT), np.float32)).astype(np.float32)
    y = np.zeros_like(x)
    return synth._cast(x.astype(np.float64), dt), synth._cast(y.astype(np.float64), dt), NT


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("variant", [0, 1])
def test_cancelling_aug_tiles_keep_relative_accuracy(ctx, orc, dt, variant):
    """Where augLISI cancels (|aug| < r/16) the combine is redone in FP64: on
    exactly summable tiles aug matches the oracle to 1e-6 relative, including
    aug = C / (m + C) which an FP32 combine rounds to 0."""
    from paper_2501_10653_gb300 import iqa
    x, y, NT = _cancelling_pair(dt)
    N = x.shape[0]
    code = parity.dtype_code(x)
    cfg = dict(variant=variant, threads=128, tiles_across=1)
    if variant == 1:
        cfg.update(stages=4, stage_kb=4)
    iqa.iqa_set_config(ctx, code, N, NT, iqa.MAPS_BOTH, cfg)
    try:
        gl, ga, gs = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    finally:
        iqa.iqa_set_config(ctx, code, N, NT, iqa.MAPS_BOTH, None)
    ol, oa, osum = parity.oracle_maps(orc, x, y, NT, PARAMS)
    assert np.array_equal(gs[:, 1:], osum[:, 1:])  # B, Sx, Sy exact
    o = oa.ravel()
    assert np.all(np.abs(o) < 0.05) and o.min() < 0 < o.max()
    assert np.all(np.abs(ga.ravel() - o) <= 1e-6 * np.abs(o))
    parity.assert_parity((gl, ga, gs), (ol, oa, osum), PARAMS)


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("N,NT", [(64, 1), (64, 2), (63, 3), (7, 7), (1, 1), (5, 1), (30, 15)])
def test_degenerate_tile_sizes(ctx, orc, dt, N, NT):
    """One-pixel and two-pixel tiles, odd sizes, a one-pixel image: random
    pixels with negatives, exact zeros and a NaN, against the oracle."""
    rng = np.random.default_rng(N * 100 + NT)
    x = rng.normal(0.0, 1.0, (N, N))
    y = rng.normal(0.0, 1.0, (N, N))
    x[0, 0] = 0.0
    if N > 2:
        y[1, 2] = np.nan
        x[N - 1, N - 1] = -0.0
    x, y = synth._cast(x, dt), synth._cast(y, dt)
    got = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    parity.assert_parity(got, parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)


def test_empty_batches_rejected(ctx):
    import torch
    from paper_2501_10653_gb300 import iqa
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_plan_create(ctx, [], iqa.IQA_F32, PARAMS)
    assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_batch_noalloc([], iqa.IQA_F32, PARAMS, torch.cuda.current_stream())
    assert ei.value.status == iqa.IQA_ERR_INVALID_ARG


def _near_equal_pair(dt):
    """A 5 x 5-tile image whose tile column c holds pixel pairs that differ by
    delta_c = 0, one storage ulp, C1/2, C1 and 1000 C1 (each y rounded to the
    storage type, so the smallest steps may round back to zero): the LISI
    denominator |x' - y'| + C1 from exactly C1 upward."""
    NT, n = 32, 5
    N = NT * n
    rng = np.random.default_rng(11)
    x = synth._cast(rng.uniform(1e-3, 1.0, (N, N)), dt)
    xs = parity.widen(x).astype(np.float64)
    col = np.arange(N) // NT
    C1 = PARAMS["C1"]
    y = synth._cast(xs + np.array([0.0, 0.0, 0.5 * C1, C1, 1e3 * C1])[col][None, :], dt)
    ulp = col == 1
    if dt == "bf16":
        y[:, ulp] = x[:, ulp] + np.uint16(1)  # next bf16 up (positive values)
    else:
        y[:, ulp] = np.nextafter(x[:, ulp], np.array(np.inf, x.dtype))
    return x, y, NT


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("variant", [0, 1])
def test_lisi_near_zero_denominator(ctx, orc, dt, variant):
    """LISI's per-pixel denominator |x' - y'| + C1 adds two nonnegative
    numbers, so FP32 keeps its relative error at one rounding however small
    |x' - y'| is (|x' - y'| itself is exact for x', y' within a factor 2):
    tiles of equal, one-ulp-apart and C1-apart pixels match the oracle to the
    FP32 tolerance with no FP64 in the per-pixel path."""
    from paper_2501_10653_gb300 import iqa
    x, y, NT = _near_equal_pair(dt)
    N = x.shape[0]
    d = np.abs(parity.widen(x).astype(np.float64) - parity.widen(y).astype(np.float64))
    assert d[:, :NT].max() == 0.0 and d[:, NT:2 * NT].min() > 0.0
    code = parity.dtype_code(x)
    cfg = dict(variant=variant, threads=128, tiles_across=1)
    if variant == 1:
        cfg.update(stages=4, stage_kb=4)
    iqa.iqa_set_config(ctx, code, N, NT, iqa.MAPS_BOTH, cfg)
    try:
        got = parity.gpu_maps(ctx, x, y, NT, PARAMS)
    finally:
        iqa.iqa_set_config(ctx, code, N, NT, iqa.MAPS_BOTH, None)
    parity.assert_parity(got, parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)


FLT_MIN = float(np.finfo(np.float32).tiny)


@pytest.mark.parametrize("variant", [0, 1])
def test_smallest_accepted_c1(ctx, orc, variant):
    """C1 must be at least the smallest normal float32: the per-pixel divide of
    Eq. 1 runs in float32 with a reciprocal that flushes subnormals.  At
    exactly that C1 (and D = C1/2, a subnormal float32) the maps match the
    oracle, with equal pixel pairs whose terms are s / C1; any smaller C1 is
    rejected before anything is launched."""
    import torch
    from paper_2501_10653_gb300 import iqa
    rng = np.random.default_rng(41)
    N, NT = 128, 32
    x = rng.uniform(-2e-16, 1e-15, (N, N)).astype(np.float32)
    y = rng.uniform(-2e-16, 1e-15, (N, N)).astype(np.float32)
    y[:, ::3] = x[:, ::3]
    p = {"C1": FLT_MIN, "C2": FLT_MIN, "C": FLT_MIN, "D": 0.0}
    cfg = dict(variant=variant, threads=128, tiles_across=1)
    if variant == 1:
        cfg.update(stages=4, stage_kb=4)
    iqa.iqa_set_config(ctx, iqa.IQA_F32, N, NT, iqa.MAPS_BOTH, cfg)
    try:
        got = parity.gpu_maps(ctx, x, y, NT, p)
    finally:
        iqa.iqa_set_config(ctx, iqa.IQA_F32, N, NT, iqa.MAPS_BOTH, None)
    parity.assert_parity(got, parity.oracle_maps(orc, x, y, NT, p), p)
    d = torch.zeros(64 * 64, device="cuda")
    m = torch.full((16,), float("nan"), device="cuda")
    for c1 in (float(np.nextafter(np.float32(FLT_MIN), np.float32(0))), FLT_MIN * (1 - 1e-9)):
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_both(ctx, d, d, iqa.IQA_F32, 64, 16, dict(p, C1=c1), m, None)
        assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert np.all(np.isnan(m.cpu().numpy()))


def test_auglisi_localises_dropped_sources(ctx, paper):
    """The paper-level behaviour on the CUDA maps: the dropped sources' tiles
    are exactly the lowest augLISI values of the paper-scale pair."""
    import test_paper_behaviour as pb
    l, a, _ = parity.gpu_maps(ctx, paper[0], paper[1], pb.NT, PARAMS)
    pb.check_localisation(l, a)


@pytest.mark.parametrize("dt", ["f32", "f16"])
def test_independent_calls_back_to_back(ctx, orc, dt):
    """IQA_OPT_INDEPENDENT_CALLS: each one-pair call loads and reduces its
    pixels while the kernel before it drains, and waits for that kernel only
    before writing.  Calls over distinct pairs (one-tile units, two-tile
    units, 256-thread CTAs and a cluster-split tile), back to back three
    times into NaN-filled maps: every map written, bit-identical to the same
    calls stream-ordered, which match the oracle."""
    import torch
    from paper_2501_10653_gb300 import iqa
    specs = [(1024, 64), (2048, 64), (2048, 128), (512, 256), (1024, 32)]
    pairs = [synth.paper_pair(pair_index=i, N=N, dtype=dt) for i, (N, _) in enumerate(specs)]
    dev = [(parity.to_device(x), parity.to_device(y)) for x, y in pairs]

    def outputs():
        return [(torch.full(((N // NT) ** 2,), float("nan"), device="cuda"),
                 torch.full(((N // NT) ** 2,), float("nan"), device="cuda"),
                 torch.full(((N // NT) ** 2, 4), float("nan"), device="cuda",
                            dtype=torch.float64)) for N, NT in specs]

    def run_all(outs, rounds):
        st = torch.cuda.current_stream()
        for _ in range(rounds):
            for (N, NT), (dx, dy), o in zip(specs, dev, outs):
                iqa.iqa_both(ctx, dx, dy, parity.dtype_code(pairs[0][0]), N, NT, PARAMS, o[0],
                             o[1], o[2], st)
        torch.cuda.synchronize()
        return [tuple(t.cpu().numpy() for t in o) for o in outs]

    want = run_all(outputs(), 1)
    for (N, NT), (x, y), w in zip(specs, pairs, want):
        parity.assert_parity(w, parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)
    iqa.iqa_set_option(ctx, iqa.IQA_OPT_INDEPENDENT_CALLS, 1)
    try:
        got = run_all(outputs(), 3)
    finally:
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INDEPENDENT_CALLS, 0)
    for g, w in zip(got, want):
        for u, v in zip(g, w):
            assert np.array_equal(u, v)
    with pytest.raises(iqa.IqaError):
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INDEPENDENT_CALLS, 2)
