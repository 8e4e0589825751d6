"""Plant plausible mistakes in a copy of the oracle and check that the pins catch
every one (no GPU).  This shows the pins constrain each part of Eq. 1 - Eq. 4:
a dropped constant, a wrong sign, a missed clamp, a transposed tile index, a
swapped sum or an off-by-one tile loop all fail at least one pin.
"""
import os
import types

import numpy as np
import pytest

import oracle
from oracle import build as obuild
import pins

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "iqa_oracle.c")).read()
AGG_SRC = open(oracle.__file__).read()

# (name, original text, planted mistake)
C_MUTANTS = [
    ("drop_C1", "A += s / (d + C1);", "A += s / (d + 1e-300);"),
    ("minus_for_plus", "double s = fabs(xi + yi);", "double s = fabs(xi - yi);"),
    ("plus_for_minus", "double d = fabs(xi - yi);", "double d = fabs(xi + yi);"),
    ("no_clamp", "return v > 0.0f ? (double)v : 0.0;", "return (double)v;"),
    ("nan_kept", "return v > 0.0f ? (double)v : 0.0;",
     "return v < 0.0f ? 0.0 : (double)v;"),
    ("transposed_tiles", "long idx = (r * NT + i) * N + (c * NT + j);",
     "long idx = (c * NT + i) * N + (r * NT + j);"),
    ("short_tile_row", "for (long j = 0; j < NT; ++j)",
     "for (long j = 0; j < NT - 1; ++j)"),
    ("max_to_min", "fmax(Sx, Sy)", "fmin(Sx, Sy)"),
    ("drop_C2", "(fmax(Sx, Sy) + C2)", "(fmax(Sx, Sy))"),
    ("drop_C", "(Sx + Sy + C)", "(Sx + Sy)"),
    ("drop_D", "D * A /", "A /"),
    ("B_squares_s", "B += s * d;", "B += s * s;"),
    ("Sx_from_y", "Sx += xi;", "Sx += yi;"),
    ("aug_no_one_minus", "aug[t] = 1.0 - B / (Sx + Sy + C);",
     "aug[t] = B / (Sx + Sy + C);"),
    ("C1_in_numerator", "A += s / (d + C1);", "A += (s + C1) / (d + C1);"),
]

AGG_MUTANTS = [
    ("eq4_no_nminus1_C", "- (n - 1) * C)", ")"),
    ("eq4_n_C", "- (n - 1) * C)", "- n * C)"),
    ("eq3_no_C2_tile", "(np.maximum(sx_t, sy_t) + C2)", "np.maximum(sx_t, sy_t)"),
    ("eq3_min", "(max(sx, sy) + C2)", "(min(sx, sy) + C2)"),
    ("merge_transposed", "blk = (slice(R * m, R * m + m), slice(Cc * m, Cc * m + m))",
     "blk = (slice(Cc * m, Cc * m + m), slice(R * m, R * m + m))"),
]


def test_real_oracle_passes_all_pins(orc):
    assert pins.run_all(orc, oracle) == []


@pytest.mark.parametrize("name,orig,bad", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_mutant_is_caught(tmp_path, name, orig, bad):
    assert SRC.count(orig) >= 1, "mutation site vanished: %s" % name
    path = obuild.build_from_source(SRC.replace(orig, bad),
                                    str(tmp_path / ("mut_%s.so" % name)))
    mut = oracle.Oracle(path)
    failed = pins.run_all(mut, oracle)
    assert failed, "planted mistake %s passed every pin" % name


@pytest.mark.parametrize("name,orig,bad", AGG_MUTANTS, ids=[m[0] for m in AGG_MUTANTS])
def test_aggregation_mutant_is_caught(orc, name, orig, bad):
    assert AGG_SRC.count(orig) == 1, "mutation site vanished: %s" % name
    mod = types.ModuleType("oracle_mut_" + name)
    mod.__dict__["np"] = np
    code = AGG_SRC.replace(orig, bad)
    # only the pure-Python aggregation functions are needed from the copy
    start = code.index("def whole_from_tiles")
    exec(compile(code[start:], "oracle_mut", "exec"), mod.__dict__)
    with pytest.raises(AssertionError):
        pins.check_eq3_eq4(orc, mod)
