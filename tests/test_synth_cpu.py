"""The host mirror of the device epoch generator (no GPU): its window form
equals the full render bit for bit, and its noise has the stated law."""
import numpy as np
import pytest

from paper_2501_10653_gb300 import synth


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_window_render_equals_full_render(dt):
    cat = synth.serving_catalog(512, 3)
    kw = dict(drop=[1, 2], add=(0, 100, 300, 0.7), dtype=dt)
    full = synth.render_epoch(cat, 123456789012, **kw)
    rng = np.random.default_rng(5)
    wins = [(0, 64, 0, 64), (448, 512, 448, 512), (37, 101, 5, 77), (511, 512, 0, 512)]
    for _ in range(6):
        r0, c0 = rng.integers(0, 500, 2)
        wins.append((int(r0), int(r0) + 12, int(c0), int(c0) + 9))
    for r0, r1, c0, c1 in wins:
        w = synth.render_epoch_window(cat, 123456789012, r0, r1, c0, c1, **kw)
        want = np.ascontiguousarray(full[r0:r1, c0:c1])
        assert np.array_equal(w.view(np.uint8), want.view(np.uint8)), (r0, c0)


def test_noise_law():
    """z = (byte sum - 510) sqrt(3)/256: mean 0, variance 1 - 2^-16, bounded by
    sqrt(12); four pixels per Philox call, so neighbours are independent."""
    z = synth.epoch_noise(512, 99).astype(np.float64).ravel()
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - (1 - 2.0**-16)) < 1e-2
    assert np.abs(z).max() <= np.sqrt(12.0)
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 1e-2
    # distinct seeds give distinct noise; the same seed the same noise
    assert not np.array_equal(synth.epoch_noise(64, 1), synth.epoch_noise(64, 2))
    assert np.array_equal(synth.epoch_noise(64, 7), synth.epoch_noise(64, 7))
