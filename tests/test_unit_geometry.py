"""The batched kernel's unit geometry, from the library's own host rules (no GPU):
for every shape a plan can take, the units it streams a pair in (TX whole tiles
across, RH tile rows down, from iqa_plan_unit_shape) cover every tile of the
pair exactly once, in image-row order, with the kernel's index arithmetic
restated here (unit -> band and column -> first tile -> tile rows and columns),
within the unit size asked for, the TMA box rules and the kernel's reduction
slots."""
import numpy as np
import pytest

from paper_2501_10653_gb300 import iqa

SIZES = (256, 288, 384, 512, 768, 1008, 1024, 2048)
TILES = (4, 8, 12, 16, 24, 32, 48, 64, 128, 256)
UNITS_KPX = (4, 16, 32, 64, 128)


def _pow2(v):
    return v > 0 and v & (v - 1) == 0


def _shape(dtype, N, NT, threads, kpx):
    cfg = {"threads": threads, "unit_kpx": kpx, "stages": 2, "stage_kb": 16, "ctas_per_sm": 1}
    try:
        return iqa.iqa_plan_unit_shape(dtype, N, NT, cfg)
    except iqa.IqaError as e:
        assert e.status == iqa.IQA_ERR_INVALID_ARG
        return None


def _check(es, N, NT, threads, kpx, TX, RH, units):
    V = 16 // es
    T = N // NT
    assert T % TX == 0 and T % RH == 0
    assert units == (T // RH) * (T // TX)
    # within the unit size asked for (a unit is at least one tile)
    unit_px = kpx * 1024
    assert TX == 1 or TX * NT * NT <= unit_px
    assert RH == 1 or RH * TX * NT * NT <= unit_px
    # a unit row is one TMA box: <= 256 elements, or whole 256-element
    # segments (up to 1024) of an image whose side is a multiple of 256
    BW = TX * NT
    assert BW <= 256 or (BW % 256 == 0 and BW <= 1024 and N % 256 == 0)
    LPU, LPT = BW // V, NT // V
    if TX > 1:
        assert threads % LPU == 0  # each consumer thread owns one column
    if RH > 1:
        # several tile rows only with the segmented reduction, whose per-row
        # slots (row groups x tiles) fit the kernel's 2 x threads
        assert TX > 1 and _pow2(LPT) and LPT <= 32 and (LPU >= 32 or _pow2(LPU))
        spr = threads // max(LPU, 32) * TX
        assert RH * spr <= 2 * threads
    # the kernel's mapping: unit lu -> band lu // units_x, column lu % units_x;
    # first tile band * RH * T + column * TX; tile (r, c) of the unit at
    # first + r * T + c, image rows band * RH * NT + r * NT, columns
    # column * TX * NT + c * NT
    units_x = T // TX
    lu = np.arange(units, dtype=np.int64)
    band, col = lu // units_x, lu % units_x
    first = band * RH * T + col * TX
    r = np.arange(RH, dtype=np.int64)[:, None]
    c = np.arange(TX, dtype=np.int64)[None, :]
    tiles = (first[:, None, None] + r * T + c).ravel()
    counts = np.bincount(tiles, minlength=T * T)
    assert counts.size == T * T and np.all(counts == 1)
    rows = (band[:, None, None] * RH * NT + r * NT + 0 * c).ravel()
    cols = (col[:, None, None] * TX * NT + 0 * r + c * NT).ravel()
    assert np.array_equal(tiles // T * NT, rows) and np.array_equal(tiles % T * NT, cols)
    # chunks stay inside the image: the unit's last row
    assert (band.max() + 1) * RH * NT <= N and (col.max() + 1) * BW <= N


@pytest.mark.parametrize("dt,es", [(iqa.IQA_F32, 4), (iqa.IQA_F16, 2), (iqa.IQA_BF16, 2)])
@pytest.mark.parametrize("threads", [128, 256, 512])
def test_units_cover_every_tile_once(dt, es, threads):
    n_ok = n_rows = 0
    for N in SIZES:
        for NT in TILES:
            for kpx in UNITS_KPX:
                got = _shape(dt, N, NT, threads, kpx)
                if got is None:
                    continue
                TX, RH, units = got
                _check(es, N, NT, threads, kpx, TX, RH, units)
                n_ok += 1
                n_rows += RH > 1
    assert n_ok > 100 and n_rows > 20


def test_paper_sizes_take_several_rows():
    """At the paper's N = 2048 the small tiles get units as large as a 64-tile
    unit: N_T = 16 FP32 takes 32 tiles x 4 rows, FP16 at its 128K default 64
    tiles x 4 rows; N_T = 64 FP16 16 tiles x 2 rows."""
    assert iqa.iqa_plan_unit_shape(iqa.IQA_F32, 2048, 16, {"unit_kpx": 32}) == (32, 4, 128)
    assert iqa.iqa_plan_unit_shape(iqa.IQA_F16, 2048, 16, {"unit_kpx": 128}) == (64, 4, 64)
    assert iqa.iqa_plan_unit_shape(iqa.IQA_F16, 2048, 64, {"unit_kpx": 128}) == (16, 2, 32)
    assert iqa.iqa_plan_unit_shape(iqa.IQA_F32, 2048, 64, {"unit_kpx": 32}) == (8, 1, 128)


def test_unit_shape_rejects_bad_arguments():
    for dtype, N, NT, cfg in ((iqa.IQA_F32, 2048, 6, {}), (iqa.IQA_F32, 2048, 512, {}),
                              (iqa.IQA_F16, 2048, 4, {}), (7, 2048, 64, {}),
                              (iqa.IQA_F32, 2048, 64, {"unit_kpx": 0}),
                              (iqa.IQA_F32, 2048, 64, {"variant": 0}),
                              (iqa.IQA_F32, 2048, 64, {"threads": 96})):
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_plan_unit_shape(dtype, N, NT, cfg)
        assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
        assert iqa.lib().iqa_last_error(None)
