"""The storage-error bound of FP16 / BF16 pixel storage (oracle.storage_bound)
against what the rounding really does (no GPU).

The bound claims: for FP32 originals x, y, the exact Eq. 1 / Eq. 2 tile values
computed from the pixels rounded to FP16 or BF16 differ from those computed
from the originals by at most the per-tile bound.  Checked here against the
FP64 oracle run on both inputs (its own rounding, about 1e-16 relative, is far
below the bounds' 1e-9 slack), on the cases where a weaker bound breaks:
* pixel pairs that rounding makes exactly equal (|x - y| collapses to 0, so
  the LISI term jumps from s / (d + C1) to s / C1: a first-order bound, with
  the denominator's own shift left out, fails here);
* FP16 subnormals (absolute, not relative, rounding error);
* zeros, negatives and NaN (the clamp commutes with rounding);
* random skies of every workload shape.
"""
import numpy as np
import pytest

from oracle import storage_bound as sb
from paper_2501_10653_gb300 import synth

P = dict(C1=1e-6, C2=1e-6, C=1e-6, D=0.5e-6)


def widen(a):
    if a.dtype == np.uint16:
        return (a.astype(np.uint32) << 16).view(np.float32)
    return a.astype(np.float32)


def rounded(v32, storage):
    return widen(synth._cast(np.asarray(v32, np.float32).astype(np.float64), storage))


def exact_change(orc, x32, y32, NT, storage, p=P):
    """|Eq. 1| and |Eq. 2| change per tile: oracle on the rounded pixels against
    the oracle on the originals."""
    args = (p["C1"], p["C2"], p["C"], p["D"])
    l0, a0, _ = orc.maps(x32, y32, NT, *args)
    l1, a1, _ = orc.maps(rounded(x32, storage), rounded(y32, storage), NT, *args)
    return np.abs(l1 - l0).ravel(), np.abs(a1 - a0).ravel(), l0.ravel(), a0.ravel()


def assert_bounded(orc, x32, y32, NT, storage, p=P):
    dl, da, l0, a0 = exact_change(orc, x32, y32, NT, storage, p)
    lb, ab, lisi, aug = sb.tile_bounds(x32, y32, NT, storage, p["C1"], p["C2"], p["C"],
                                       p["D"])
    # the bound's own FP64 values of Eq. 1 / Eq. 2 are the oracle's
    assert np.allclose(lisi, l0, rtol=1e-12, atol=0)
    assert np.allclose(aug, a0, rtol=1e-12, atol=1e-15)
    assert np.all(dl <= lb), (storage, np.max(dl - lb))
    assert np.all(da <= ab), (storage, np.max(da - ab))
    return dl, da, lb, ab


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_tie_collapses_difference(orc, storage):
    """One pixel pair: x = 1 + u_s (exactly halfway between 1 and the next
    stored value, so it rounds to the even neighbour 1.0) and y = 1.  Rounded,
    the pair is equal and the LISI term becomes s / C1."""
    u = sb.STORAGE[storage][0]
    x = np.array([[1.0 + u]], np.float32)
    y = np.array([[1.0]], np.float32)
    assert rounded(x, storage)[0, 0] == 1.0
    dl, da, lb, ab = assert_bounded(orc, x, y, 1, storage)
    # the exact values, by hand: originals s = 2 + u, d = u; rounded s = 2, d = 0
    C1, C2, C, D = P["C1"], P["C2"], P["C"], P["D"]
    l_orig = D * (2 + u) / (u + C1) / ((1 + u) + C2)
    l_round = D * 2 / C1 / (1 + C2)
    assert dl[0] == pytest.approx(abs(l_round - l_orig), rel=1e-12)
    a_orig = 1 - (2 + u) * u / ((2 + u) + C)
    assert da[0] == pytest.approx(abs(1.0 - a_orig), rel=1e-12)
    # the jump is orders of magnitude above the rounding itself ...
    assert dl[0] / l_orig > 100
    # ... and a first-order bound, blind to the denominator falling to C1,
    # would miss it: es (t + s) / t^2 summed with the original t
    es = sb.pixel_error(np.float64(1.0 + u), storage) + sb.pixel_error(np.float64(1.0),
                                                                        storage)
    t, s = u + C1, 2 + u
    first_order = D * (es * (t + s) / (t * t) * ((1 + u) + C2) + (2 + u) / t * es) / \
        ((1 + u) + C2) ** 2
    assert first_order < dl[0] <= lb[0]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_near_equal_noise(orc, storage):
    """Tiles of nearly equal pixel pairs at the noise level, where the storage
    spacing exceeds C1: the regime in which the LISI bound is loose but must
    still hold."""
    rng = np.random.default_rng(11)
    x = (5e-3 * rng.standard_normal((64, 64))).astype(np.float32)
    y = (x + 1e-7 * rng.standard_normal((64, 64))).astype(np.float32)
    dl, da, lb, ab = assert_bounded(orc, x, y, 16, storage)
    assert np.max(dl) > 0


def test_fp16_subnormals_and_specials(orc):
    """FP16 subnormals (absolute rounding error up to 2^-25), zeros, negatives,
    NaN and pixels that round up into the normal range."""
    rng = np.random.default_rng(5)
    x = rng.uniform(-2e-5, 6.2e-5, (32, 32)).astype(np.float32)
    y = rng.uniform(-2e-5, 6.2e-5, (32, 32)).astype(np.float32)
    x[::7, ::5] = 0.0
    y[::3, ::4] = np.nan
    x[1, :] = -1.0
    y[2, 3] = 6.1e-5
    for NT in (1, 4, 32):
        assert_bounded(orc, x, y, NT, "f16")
        assert_bounded(orc, x, y, NT, "bf16")


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_other_constants(orc, storage):
    rng = np.random.default_rng(8)
    x = rng.uniform(-0.2, 1.0, (32, 32)).astype(np.float32)
    y = (x + rng.normal(0, 1e-3, (32, 32))).astype(np.float32)
    for p in (dict(C1=1e-3, C2=1e-4, C=1e-2, D=0.0),
              dict(C1=1e-8, C2=1e-6, C=1e-6, D=2e-7),
              dict(C1=2.0 ** -20, C2=0.5, C=0.0, D=0.0)):
        q = dict(p)
        if q["D"] <= 0:
            q["D"] = q["C1"] / 2
        assert_bounded(orc, x, y, 8, storage, q)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_sky_workloads(orc, storage):
    """The small pair (N=256) and one paper-scale pair (N=2048) at every tile
    size of the paper's sweep."""
    x, y = synth.small_pair()
    assert_bounded(orc, x, y, 64, storage)
    x, y = synth.paper_pair()
    for NT in (16, 64, 256):
        assert_bounded(orc, x, y, NT, storage)


def test_fp32_storage_has_zero_change(orc):
    x, y = synth.small_pair()
    dl, da, lb, ab = assert_bounded(orc, x, y, 64, "f32")
    assert np.all(dl == 0) and np.all(da == 0)


def test_rejects_out_of_range_pixels():
    x = np.full((4, 4), 7e4, np.float32)
    with pytest.raises(ValueError):
        sb.tile_bounds(x, x, 2, "f16", 1e-6, 1e-6, 1e-6)
    sb.tile_bounds(x, x, 2, "bf16", 1e-6, 1e-6, 1e-6)


def test_zero_constants_give_infinite_bounds_only_where_needed():
    x = np.zeros((4, 4), np.float32)
    y = np.zeros((4, 4), np.float32)
    y[0, 0] = 1.0
    lb, ab, _, _ = sb.tile_bounds(x, y, 2, "f16", 1e-6, 0.0, 0.0)
    # tile 0 holds a nonzero pixel; the all-zero tiles may round to all-zero
    # sums, where C2 = C = 0 leaves no lower bound on the denominators
    assert np.isfinite(lb[0]) and np.isfinite(ab[0])
    assert np.all(np.isinf(lb[1:])) and np.all(np.isinf(ab[1:]))
