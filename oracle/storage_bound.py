"""Storage-error bound of the per-tile LISI / augLISI values when the pixels are
stored in FP16 or BF16 instead of FP32 (TEST INFRASTRUCTURE ONLY: imported by
``tests/`` and by the benchmark's CPU-baseline leg; it shares no code with the
CUDA library and never imports it).

What it bounds.  Let x, y be the FP32 originals and x~, y~ the same pixels
rounded to nearest in the storage type.  Eq. 1 and Eq. 2 (Section 2) computed
exactly from x~, y~ differ from the same equations computed exactly from x, y;
``tile_bounds`` returns, per tile, an upper bound on that difference, computed
from the originals alone (it never looks at the rounded pixels, so it is a
guarantee for any input, not a measurement).

Derivation (every step an inequality, no first-order truncation):

* Clamp and rounding commute: rounding to nearest is monotone and maps 0 to 0,
  so round(max(v, 0)) = max(round(v), 0) (a negative or NaN pixel reads as 0
  either way).  For a clamped original v >= 0 the stored value differs by at
  most e(v) = 0 if v == 0, else max(u_s v, eta_s), with the unit roundoff
  u_s = 2^-11 (FP16) or 2^-8 (BF16) and eta_s half the spacing of the
  subnormals (2^-25 for FP16, 2^-134 for BF16).  The originals must be finite
  and below the largest finite value of the storage type (65504 for FP16).
* Per pixel, s = x + y and t = |x - y| + C1 move by at most
  es = e(x) + e(y) each (|x~ - y~| - |x - y| is at most |dx - dy|), and the
  stored denominator is at least t_min = max(C1, t - es).  Then
    |s~/t~ - s/t| = |ds t - s dt| / (t t~) <= es (t + s) / (t t_min)     (Eq. 1)
    |s~ d~ - s d| <= es d + s es + es^2,  d = |x - y|                    (Eq. 2)
  and |dSx| <= sum e(x), |dSy| <= sum e(y) over the tile.
* LISI = D A / M with M = max(Sx, Sy) + C2: |dM| <= EM = max(sum e(x),
  sum e(y)) (max is 1-Lipschitz in each argument), so
    |dLISI| <= D (EA M + A EM) / (M max(C2, M - EM)),   EA = bound on |dA|.
* augLISI = 1 - B / Q with Q = Sx + Sy + C: |dQ| <= EQ = sum e(x) + e(y), so
    |dAug| = |d(B/Q)| <= (EB Q + B EQ) / (Q max(C, Q - EQ)).
* A bound is reported as +inf when a denominator's lower bound is 0 (C2 = 0 or
  C = 0 on a tile whose sums may round to 0).

Where it is vacuous.  The LISI term's relative change is about es / t_min:
where the storage spacing of a pixel (u_s times its value) reaches |x - y| +
C1, nearly equal pixel pairs can change their term by more than 100%, and the
bound on such tiles is of the order of the terms themselves.  With C1 = 1e-6
that happens for FP16 pixels above about 2e-3 and BF16 pixels above about
2.6e-4, which includes the noise floor of the precision workload; augLISI,
whose per-pixel term s d vanishes as x -> y, has no such amplification.

The arithmetic here is FP64 over per-pixel arrays; its own rounding (relative
1e-15) is covered by the factor (1 + 1e-9) applied to every bound.
"""
import numpy as np

#: unit roundoff and half the subnormal spacing of each storage type
STORAGE = {
    "f32": (2.0 ** -24, 2.0 ** -150),
    "f16": (2.0 ** -11, 2.0 ** -25),
    "bf16": (2.0 ** -8, 2.0 ** -134),
}
#: largest finite value of each storage type
STORAGE_MAX = {"f32": 3.4028234663852886e38, "f16": 65504.0, "bf16": 3.3895313892515355e38}

_SLACK = 1.0 + 1e-9


def _clamped(v):
    v = np.asarray(v, dtype=np.float64)
    return np.where(v > 0.0, v, 0.0)  # NaN -> 0 as well (Section 2 clamp)


def pixel_error(v, storage):
    """e(v): the largest change that rounding the clamped original v >= 0 to
    the storage type can make (0 for v == 0)."""
    u, eta = STORAGE[storage]
    return np.where(v > 0.0, np.maximum(u * v, eta), 0.0)


def tile_bounds(x, y, NT, storage, C1, C2, C, D=None, band_rows=None):
    """Per-tile bounds (lisi_bound, aug_bound), FP64 arrays of (N/NT)^2 values
    in tile order t = r (N/NT) + c, plus the FP64 per-tile values of Eq. 1 and
    Eq. 2 on the originals that the bound is relative to (lisi, aug).

    x, y: N x N FP32 originals (before rounding and clamping).  D <= 0 or None
    means C1 / 2 (the default constant of the library)."""
    x = np.asarray(x)
    y = np.asarray(y)
    N = x.shape[0]
    if x.shape != (N, N) or y.shape != (N, N) or N % NT:
        raise ValueError("need N x N images with NT dividing N")
    if D is None or D <= 0.0:
        D = C1 / 2.0
    top = STORAGE_MAX[storage]
    if not (np.all(np.abs(np.nan_to_num(x, nan=0.0)) < top) and
            np.all(np.abs(np.nan_to_num(y, nan=0.0)) < top)):
        raise ValueError("pixels beyond the storage type's finite range")
    T = N // NT
    band = band_rows or max(NT, (1 << 22) // N // NT * NT)
    sums = {k: np.zeros(T * T) for k in ("A", "B", "Sx", "Sy", "EA", "EB", "ex", "ey")}
    for r0 in range(0, N, band):
        r1 = min(N, r0 + band)
        xb = _clamped(x[r0:r1])
        yb = _clamped(y[r0:r1])
        ex = pixel_error(xb, storage)
        ey = pixel_error(yb, storage)
        es = ex + ey
        s = xb + yb
        d = np.abs(xb - yb)
        t = d + C1
        tmin = np.maximum(C1, t - es)
        parts = {
            "A": s / t,
            "B": s * d,
            "Sx": xb,
            "Sy": yb,
            "EA": es * (t + s) / (t * tmin),
            "EB": es * d + s * es + es * es,
            "ex": ex,
            "ey": ey,
        }
        lo, hi = (r0 // NT) * T, (r1 // NT) * T
        for k, a in parts.items():
            sums[k][lo:hi] += _tile_sum_rows(a, NT, T)
    A, B, Sx, Sy = sums["A"], sums["B"], sums["Sx"], sums["Sy"]
    M = np.maximum(Sx, Sy) + C2
    Q = Sx + Sy + C
    EM = np.maximum(sums["ex"], sums["ey"])
    EQ = sums["ex"] + sums["ey"]
    Mmin = np.maximum(C2, M - EM)
    Qmin = np.maximum(C, Q - EQ)
    with np.errstate(divide="ignore", invalid="ignore"):
        lisi = D * A / M
        aug = 1.0 - B / Q
        lb = D * (sums["EA"] * M + A * EM) / (M * Mmin)
        ab = (sums["EB"] * Q + B * EQ) / (Q * Qmin)
    lb = np.where(Mmin > 0.0, lb, np.inf) * _SLACK
    ab = np.where(Qmin > 0.0, ab, np.inf) * _SLACK
    return lb, ab, lisi, aug


def _tile_sum_rows(a, NT, T):
    """Per-tile sums of a band of whole tile rows (rows x N array)."""
    rows = a.shape[0]
    return a.reshape(rows // NT, NT, T, NT).sum(axis=(1, 3)).ravel()
