"""Exact-rational brute force of Eq. 1 and Eq. 2 for tiny images (test infrastructure).

Every operation in Eq. 1 and Eq. 2 (Section 1) is +, -, |.|, / or max, so with
rational inputs the per-tile LISI and augLISI are exact rationals.  This module
evaluates them with ``fractions.Fraction`` and pure-Python loops, so it has no
rounding at all; the FP64 oracle must agree with it to FP64 rounding.  The
clamp of Section 2 reads as "v > 0 ? v : 0" (NaN becomes 0).
"""
from fractions import Fraction
import math


def _clamp(v):
    """Section 2 pre-processing; a float NaN fails "v > 0" and becomes 0."""
    if isinstance(v, float) and math.isnan(v):
        return Fraction(0)
    q = Fraction(v)
    return q if q > 0 else Fraction(0)


def tile_values(x, y, NT, C1, C2, C, D):
    """Per-tile (lisi, auglisi, A, B, Sx, Sy) as Fractions, tiles in row-major
    order t = r*(N/NT) + c.  x, y: N x N nested lists (or arrays) of numbers."""
    N = len(x)
    C1, C2, C, D = Fraction(C1), Fraction(C2), Fraction(C), Fraction(D)
    per_row = N // NT
    out = []
    for r in range(per_row):
        for c in range(per_row):
            A = B = Sx = Sy = Fraction(0)
            for i in range(r * NT, r * NT + NT):
                for j in range(c * NT, c * NT + NT):
                    xi = _clamp(x[i][j])
                    yi = _clamp(y[i][j])
                    s = abs(xi + yi)
                    d = abs(xi - yi)
                    A += s / (d + C1)
                    B += s * d
                    Sx += xi
                    Sy += yi
            lisi = D * A / (max(Sx, Sy) + C2)
            aug = 1 - B / (Sx + Sy + C)
            out.append((lisi, aug, A, B, Sx, Sy))
    return out
