"""The FP64 oracle against what the paper and mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
import pins


@pytest.mark.parametrize("check", pins.ALL_ORACLE_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(orc, check):
    check(orc)


def test_eq3_eq4_identities(orc):
    pins.check_eq3_eq4(orc, oracle)


def test_golden_file_parses():
    cases = pins.load_golden()
    assert {c["name"] for c in cases} >= {"mixed_2x2", "four_tiles",
                                          "four_tiles_whole", "identical",
                                          "all_clamped"}
    for c in cases:
        assert c["cite"]


def test_bad_shapes_rejected(orc):
    x = np.zeros((8, 8), np.float32)
    with pytest.raises(ValueError):
        orc.maps(x, x, 3, 1e-6, 1e-6, 1e-6, 5e-7)
    with pytest.raises(ValueError):
        orc.tile_sums(x, x, 4, 1e-6, tiles=[4])


def test_openmp_threads_do_not_change_results(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((128, 128)).astype(np.float32)
    y = rng.standard_normal((128, 128)).astype(np.float32)
    a = orc.maps(x, y, 16, 1e-6, 1e-6, 1e-6, 5e-7, threads=1)
    b = orc.maps(x, y, 16, 1e-6, 1e-6, 1e-6, 5e-7, threads=4)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
