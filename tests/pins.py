"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics, not by
the oracle itself.

Each ``check_*`` takes an ``oracle.Oracle`` (the real one, or a planted mutant)
and raises ``AssertionError`` when the oracle disagrees with the fact.  The
aggregation checks take the module that provides ``whole_from_tiles`` and
``merge_tiles`` (Eq. 3 / Eq. 4), so a mutant of those can be checked too.

Sources of truth:
* ``tests/golden/hand_worked.txt``: hand-derived exact values (Eq. 1, Eq. 2,
  Eq. 3, Eq. 4, Section 2 clamp and tiling);
* an exact-rational brute force on tiny inputs (``oracle.exact``);
* closed forms on constant tiles, on identical inputs and on y = 0;
* properties stated in Section 1 (values in [0, 1] for inputs in [0, 1], 1 for
  identical inputs) and Section 2 (negatives set to zero), symmetry;
* the Eq. 3 / Eq. 4 identities against the whole image computed directly;
* tile markers: changing one tile changes exactly its own map entry.
"""
import os
from fractions import Fraction

import numpy as np

from oracle import exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "hand_worked.txt")


def _frac(tok):
    return Fraction(tok)


def load_golden(path=GOLDEN):
    """Parse the ``[case]`` blocks of the golden file into dicts."""
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = {"name": line[1:-1]}
                cases.append(cur)
                continue
            key, val = [s.strip() for s in line.split("=", 1)]
            cur[key] = val
    out = []
    for c in cases:
        d = {"name": c["name"], "cite": c["cite"]}
        for k in ("N", "NT"):
            d[k] = int(c[k])
        for k in ("C1", "C2", "C", "D"):
            d[k] = _frac(c[k])
        for k in ("x", "y"):
            d[k] = np.array([float(v) for v in c[k].split()], dtype=np.float32
                            ).reshape(d["N"], d["N"])
        for k in ("lisi", "aug", "A", "B", "Sx", "Sy"):
            d[k] = [_frac(v) for v in c[k].split()]
        out.append(d)
    return out


def _close(got, want, rel, what):
    want = float(want)
    tol = rel * max(1.0, abs(want))
    assert abs(got - want) <= tol, "%s: got %r want %r" % (what, got, want)


def check_golden(orc, rel=1e-13):
    """Hand-derived exact values."""
    for c in load_golden():
        lisi, aug, sums = orc.maps(c["x"], c["y"], c["NT"], float(c["C1"]),
                                   float(c["C2"]), float(c["C"]), float(c["D"]))
        lisi, aug = lisi.ravel(), aug.ravel()
        assert lisi.size == len(c["lisi"]), c["name"]
        for t in range(lisi.size):
            tag = "%s tile %d" % (c["name"], t)
            _close(lisi[t], c["lisi"][t], rel, tag + " lisi")
            _close(aug[t], c["aug"][t], rel, tag + " aug")
            for k, key in enumerate(("A", "B", "Sx", "Sy")):
                _close(sums[t, k], c[key][t], rel, tag + " " + key)


def _rand_tiny(rng, N):
    """Small dyadic values with negatives, zeros, ties and NaN."""
    x = rng.integers(-8, 17, (N, N)).astype(np.float32) / 8.0
    y = rng.integers(-8, 17, (N, N)).astype(np.float32) / 8.0
    tie = rng.random((N, N)) < 0.2
    y[tie] = x[tie]
    x[rng.random((N, N)) < 0.05] = np.nan
    y[rng.random((N, N)) < 0.05] = np.nan
    return x, y


def check_exact_bruteforce(orc, seed=11):
    """FP64 oracle within FP64 rounding of the exact rational result."""
    rng = np.random.default_rng(seed)
    C1, C2, C, D = 0.5, 0.25, 0.125, 0.25
    for N, NT in ((4, 4), (8, 4), (16, 4), (6, 3), (8, 2)):
        x, y = _rand_tiny(rng, N)
        lisi, aug, sums = orc.maps(x, y, NT, C1, C2, C, D)
        ex = exact.tile_values(x.tolist(), y.tolist(), NT, C1, C2, C, D)
        for t, (l, a, A, B, Sx, Sy) in enumerate(ex):
            r = B / (Sx + Sy + Fraction(C))
            tag = "N=%d NT=%d tile %d" % (N, NT, t)
            _close(lisi.ravel()[t], l, 1e-12, tag + " lisi")
            assert abs(aug.ravel()[t] - float(a)) <= 1e-12 * max(1.0, float(r)), tag
            for k, v in enumerate((A, B, Sx, Sy)):
                _close(sums[t, k], v, 1e-12, tag + " sum %d" % k)


def check_constant_tiles(orc):
    """Constant tile x = a, y = b over m pixels:
    lisi = D m (a+b)/(|a-b|+C1) / (m max(a,b) + C2),
    aug  = 1 - m |a^2 - b^2| / (m (a+b) + C)."""
    NT, C1, C2, C = 8, 1e-3, 2e-3, 3e-3
    D = C1 / 2
    m = NT * NT
    for a, b in ((0.25, 0.75), (1.5, 0.5), (2.0, 2.0), (0.3, 0.0), (0.0, 0.7),
                 (1e-4, 3e-4)):
        x = np.full((NT, NT), a, dtype=np.float32)
        y = np.full((NT, NT), b, dtype=np.float32)
        a64, b64 = float(np.float32(a)), float(np.float32(b))
        lisi, aug, _ = orc.maps(x, y, NT, C1, C2, C, D)
        want_l = D * m * (a64 + b64) / (abs(a64 - b64) + C1) / (m * max(a64, b64) + C2)
        want_a = 1 - m * abs(a64 * a64 - b64 * b64) / (m * (a64 + b64) + C)
        _close(lisi[0, 0], want_l, 1e-12, "constant lisi a=%g b=%g" % (a, b))
        _close(aug[0, 0], want_a, 1e-12, "constant aug a=%g b=%g" % (a, b))


def check_identical_inputs(orc, seed=12):
    """x = y: augLISI is exactly 1 and, with D = C1/2, LISI = Sx/(Sx + C2)
    (Section 1: identical images give the top value)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((32, 32)).astype(np.float32)
    C1 = C2 = C = 1e-6
    lisi, aug, sums = orc.maps(x, x, 8, C1, C2, C, C1 / 2)
    assert np.all(aug == 1.0), "augLISI of identical tiles must be exactly 1"
    sx = sums[:, 2]
    np.testing.assert_allclose(lisi.ravel(), sx / (sx + C2), rtol=1e-12)
    assert np.all(lisi <= 1.0)


def check_zero_tiles(orc):
    """All-non-positive tiles: LISI is exactly 0 and augLISI exactly 1."""
    x = -np.abs(np.random.default_rng(13).standard_normal((16, 16))).astype(np.float32)
    y = x.copy()
    y[::2] = 0.0
    y[1, 1] = np.nan
    lisi, aug, sums = orc.maps(x, y, 4, 1e-6, 1e-6, 1e-6, 5e-7)
    assert np.all(lisi == 0.0) and np.all(aug == 1.0) and np.all(sums == 0.0)


def check_y_zero(orc, seed=14):
    """y = 0: every |x - y| = |x + y| = x, so aug = 1 - sum x^2 / (sum x + C),
    and LISI = D sum x/(x + C1) / (sum x + C2)."""
    rng = np.random.default_rng(seed)
    x = rng.random((16, 16)).astype(np.float32)
    y = np.zeros_like(x)
    C1, C2, C, D = 1e-3, 1e-3, 1e-3, 5e-4
    lisi, aug, _ = orc.maps(x, y, 16, C1, C2, C, D)
    x64 = x.astype(np.float64)
    want_a = 1 - np.sum(x64 * x64) / (np.sum(x64) + C)
    want_l = D * np.sum(x64 / (x64 + C1)) / (np.sum(x64) + C2)
    _close(aug[0, 0], want_a, 1e-12, "y=0 aug")
    _close(lisi[0, 0], want_l, 1e-12, "y=0 lisi")


def check_symmetry(orc, seed=15):
    """f(x, y) = f(y, x) bit-exactly (Eq. 1 and Eq. 2 are symmetric)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((64, 64)).astype(np.float32)
    y = rng.standard_normal((64, 64)).astype(np.float32)
    l1, a1, s1 = orc.maps(x, y, 16, 1e-6, 1e-6, 1e-6, 5e-7)
    l2, a2, s2 = orc.maps(y, x, 16, 1e-6, 1e-6, 1e-6, 5e-7)
    assert np.array_equal(l1, l2) and np.array_equal(a1, a2)
    assert np.array_equal(s1[:, :2], s2[:, :2])
    assert np.array_equal(s1[:, 2], s2[:, 3]) and np.array_equal(s1[:, 3], s2[:, 2])


def check_clamp_invariance(orc, seed=16):
    """Section 2: negatives are set to zero, so replacing non-positive pixels by
    other non-positive values (or NaN) changes nothing, bit-exactly."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((64, 64)).astype(np.float32)
    y = rng.standard_normal((64, 64)).astype(np.float32)
    base = orc.maps(x, y, 16, 1e-6, 1e-6, 1e-6, 5e-7)
    x2, y2 = x.copy(), y.copy()
    nx, ny = x2 <= 0, y2 <= 0
    x2[nx] = -rng.random(nx.sum()).astype(np.float32) * 100
    y2[ny] = np.where(rng.random(ny.sum()) < 0.5, np.nan, 0.0).astype(np.float32)
    other = orc.maps(x2, y2, 16, 1e-6, 1e-6, 1e-6, 5e-7)
    for u, v in zip(base, other):
        assert np.array_equal(u, v)
    # and a clamp that is applied makes a difference when negatives are kept:
    z = np.zeros_like(x)
    l_neg, _, _ = orc.maps(-np.abs(x) - 1, z, 16, 1e-6, 1e-6, 1e-6, 5e-7)
    assert np.all(l_neg == 0.0)


def check_range(orc, seed=17):
    """Section 1: for inputs in [0, 1] both maps lie in [0, 1] (D = C1/2)."""
    rng = np.random.default_rng(seed)
    for _ in range(4):
        x = rng.random((64, 64)).astype(np.float32)
        y = np.clip(x + 0.3 * rng.standard_normal((64, 64)), 0, 1).astype(np.float32)
        C1 = C2 = C = 1e-6
        lisi, aug, _ = orc.maps(x, y, 8, C1, C2, C, C1 / 2)
        assert np.all((lisi >= 0) & (lisi <= 1)), "LISI out of [0,1]"
        assert np.all((aug >= 0) & (aug <= 1)), "augLISI out of [0,1]"


def check_eq3_eq4(orc, agg, seed=18):
    """Eq. 3 and Eq. 4: the whole image computed directly (N_T = N) equals the
    value rebuilt from its tiles; merging m x m tile blocks equals computing at
    N_T' = m N_T (Section 3: a larger tile formed by merging smaller ones)."""
    rng = np.random.default_rng(seed)
    N = 64
    x = (rng.standard_normal((N, N)) * 0.2 + 0.1).astype(np.float32)
    y = (rng.standard_normal((N, N)) * 0.2 + 0.1).astype(np.float32)
    C1, C2, C = 1e-3, 2e-3, 5e-3
    D = C1 / 2
    for NT in (4, 8, 16):
        lisi, aug, sums = orc.maps(x, y, NT, C1, C2, C, D)
        wl, wa, _ = orc.maps(x, y, N, C1, C2, C, D)
        gl, ga = agg.whole_from_tiles(lisi, aug, sums[:, 2], sums[:, 3], C2, C)
        _close(gl, wl[0, 0], 1e-12, "Eq. 3 NT=%d" % NT)
        _close(ga, wa[0, 0], 1e-12, "Eq. 4 NT=%d" % NT)
        for m in (2, 4):
            if (N // NT) % m:
                continue
            ml, ma = agg.merge_tiles(lisi, aug, sums, m, C2, C)
            bl, ba, _ = orc.maps(x, y, NT * m, C1, C2, C, D)
            np.testing.assert_allclose(ml, bl, rtol=1e-12, atol=0)
            np.testing.assert_allclose(ma, ba, rtol=1e-12, atol=1e-12)


def check_tile_markers(orc, seed=19):
    """Perturbing only tile (r, c) of y changes exactly map entry r*(N/N_T)+c."""
    rng = np.random.default_rng(seed)
    N, NT = 16, 4
    T = N // NT
    x = (rng.random((N, N)) + 0.5).astype(np.float32)
    y = x.copy()
    base_l, base_a, _ = orc.maps(x, y, NT, 1e-6, 1e-6, 1e-6, 5e-7)
    for r in range(T):
        for c in range(T):
            y2 = y.copy()
            y2[r * NT + 1, c * NT + 2] += 0.25
            l, a, _ = orc.maps(x, y2, NT, 1e-6, 1e-6, 1e-6, 5e-7)
            changed_l = np.argwhere(l.ravel() != base_l.ravel()).ravel().tolist()
            changed_a = np.argwhere(a.ravel() != base_a.ravel()).ravel().tolist()
            assert changed_l == [r * T + c], (r, c, changed_l)
            assert changed_a == [r * T + c], (r, c, changed_a)


def check_sparse_tile_list(orc, seed=20):
    """Sums for a listed subset of tiles equal the full map's rows."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((32, 32)).astype(np.float32)
    y = rng.standard_normal((32, 32)).astype(np.float32)
    _, _, sums = orc.maps(x, y, 8, 1e-6, 1e-6, 1e-6, 5e-7)
    pick = [15, 0, 7, 3]
    part = orc.tile_sums(x, y, 8, 1e-6, tiles=pick)
    assert np.array_equal(part, sums[pick])


ALL_ORACLE_CHECKS = [check_golden, check_exact_bruteforce, check_constant_tiles,
                     check_identical_inputs, check_zero_tiles, check_y_zero,
                     check_symmetry, check_clamp_invariance, check_range,
                     check_tile_markers, check_sparse_tile_list]


def run_all(orc, agg):
    """Every pin; returns the list of (name, error) that failed."""
    failed = []
    for chk in ALL_ORACLE_CHECKS:
        try:
            chk(orc)
        except (AssertionError, ValueError, ZeroDivisionError) as e:
            failed.append((chk.__name__, str(e)[:200]))
    try:
        check_eq3_eq4(orc, agg)
    except (AssertionError, ValueError, ZeroDivisionError) as e:
        failed.append(("check_eq3_eq4", str(e)[:200]))
    return failed

