"""FP64 CPU oracle for the tile-wise LISI / augLISI maps of arxiv 2501.10653.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never imports it.

Contents
--------
* ``tile_sums`` / ``maps``: Eq. 1 and Eq. 2 per tile (Section 2), computed by the
  plain C loop in ``iqa_oracle.c`` in FP64 over the clamped pixels.
* ``whole_from_tiles``: Eq. 3 and Eq. 4 (Section 3), which rebuild the value of
  the whole image -- or of a larger tile formed by merging smaller ones -- from
  the per-tile values and the per-tile pixel sums.
* ``merge_tiles``: Eq. 3 / Eq. 4 applied to every m x m block of tiles.
* ``exact``: an exact-rational brute force of Eq. 1 / Eq. 2 for tiny inputs.
* ``storage_bound``: a bound, from the FP32 originals alone, on how far Eq. 1
  and Eq. 2 move when the pixels are stored in FP16 or BF16.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(hand-derived golden values, closed forms, the Eq. 3 / Eq. 4 identities, tile
markers, invariants) and by ``tests/test_oracle_mutants.py``; the storage bound
by ``tests/test_storage_bound.py`` (against the oracle on the original and the
rounded pixels, including a hand-computed rounding tie).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load(path=None):
    lib = ctypes.CDLL(path or _build.build())
    f64p = ctypes.POINTER(ctypes.c_double)
    f32p = ctypes.POINTER(ctypes.c_float)
    i64p = ctypes.POINTER(ctypes.c_long)
    lib.iqa_oracle_tile_sums.argtypes = [f32p, f32p, ctypes.c_long, ctypes.c_long,
                                         ctypes.c_double, i64p, ctypes.c_long,
                                         f64p, ctypes.c_int]
    lib.iqa_oracle_tile_sums.restype = ctypes.c_int
    lib.iqa_oracle_maps.argtypes = [f32p, f32p, ctypes.c_long, ctypes.c_long,
                                    ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double,
                                    f64p, f64p, f64p, ctypes.c_int]
    lib.iqa_oracle_maps.restype = ctypes.c_int
    lib.iqa_oracle_has_openmp.restype = ctypes.c_int
    return lib


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


class Oracle:
    """Python face of one compiled oracle library (the real one, or a planted
    mutant in the mutation tests)."""

    def __init__(self, path=None):
        self._lib = _load(path) if path else lib()

    @property
    def has_openmp(self):
        return bool(self._lib.iqa_oracle_has_openmp())

    @staticmethod
    def _img(a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        if a.ndim != 2 or a.shape[0] != a.shape[1]:
            raise ValueError("images must be square N x N")
        return a

    def tile_sums(self, x, y, NT, C1, tiles=None, threads=1):
        """Per-tile (A, B, Sx, Sy) in FP64, shape (len(tiles) or n, 4).

        A = sum |x+y|/(|x-y|+C1) and B = sum |x+y||x-y| are the numerator sums of
        Eq. 1 and Eq. 2; Sx, Sy the clamped pixel sums of the tile.
        """
        x, y = self._img(x), self._img(y)
        N = x.shape[0]
        if y.shape != x.shape:
            raise ValueError("x and y differ in shape")
        n = (N // NT) ** 2 if NT > 0 and N % NT == 0 else 0
        if tiles is None:
            tl, count, tp = None, n, None
        else:
            tl = np.ascontiguousarray(tiles, dtype=np.int64)
            count = tl.size
            tp = tl.ctypes.data_as(ctypes.POINTER(ctypes.c_long))
        out = np.zeros((count, 4), dtype=np.float64)
        rc = self._lib.iqa_oracle_tile_sums(
            x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
            y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), N, NT, float(C1),
            tp, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            int(threads))
        if rc != 0:
            raise ValueError("bad shape or tile index (N=%d, NT=%d)" % (N, NT))
        return out

    def maps(self, x, y, NT, C1, C2, C, D, threads=1):
        """(lisi, aug, sums): the Eq. 1 and Eq. 2 maps, shape (N/NT, N/NT), FP64,
        tile t = r*(N/NT)+c at [r, c]; sums shape (n, 4)."""
        x, y = self._img(x), self._img(y)
        N = x.shape[0]
        if y.shape != x.shape:
            raise ValueError("x and y differ in shape")
        if NT < 1 or N % NT != 0:
            raise ValueError("N_T must divide N")
        m = N // NT
        lisi = np.zeros(m * m, dtype=np.float64)
        aug = np.zeros(m * m, dtype=np.float64)
        sums = np.zeros((m * m, 4), dtype=np.float64)
        f64p = ctypes.POINTER(ctypes.c_double)
        rc = self._lib.iqa_oracle_maps(
            x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
            y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), N, NT,
            float(C1), float(C2), float(C), float(D),
            lisi.ctypes.data_as(f64p), aug.ctypes.data_as(f64p),
            sums.ctypes.data_as(f64p), int(threads))
        if rc != 0:
            raise ValueError("bad shape (N=%d, NT=%d)" % (N, NT))
        return lisi.reshape(m, m), aug.reshape(m, m), sums


def whole_from_tiles(lisi_t, aug_t, sx_t, sy_t, C2, C):
    """Eq. 3 and Eq. 4 (Section 3): the LISI and augLISI of the whole region
    covered by the given tiles, rebuilt from the per-tile values and the
    per-tile clamped pixel sums, in the order the equations write them.

    Eq. 3: LISI = sum_t lisi_t * (max(Sx_t, Sy_t) + C2) / (max(Sx, Sy) + C2)
    Eq. 4: augLISI = [sum_t auglisi_t * (Sx_t + Sy_t + C) - (n - 1) C]
                     / (Sx + Sy + C)
    with Sx, Sy the sums over the whole region and n the number of tiles.
    """
    lisi_t = np.asarray(lisi_t, dtype=np.float64).ravel()
    aug_t = np.asarray(aug_t, dtype=np.float64).ravel()
    sx_t = np.asarray(sx_t, dtype=np.float64).ravel()
    sy_t = np.asarray(sy_t, dtype=np.float64).ravel()
    n = lisi_t.size
    sx = float(np.sum(sx_t))
    sy = float(np.sum(sy_t))
    lisi = float(np.sum(lisi_t * (np.maximum(sx_t, sy_t) + C2))) / (max(sx, sy) + C2)
    aug = (float(np.sum(aug_t * (sx_t + sy_t + C))) - (n - 1) * C) / (sx + sy + C)
    return lisi, aug


def merge_tiles(lisi_map, aug_map, sums, m, C2, C):
    """Maps of the larger tiles formed by merging every m x m block of tiles
    (Section 3: the "entire image" of Eq. 3 / Eq. 4 may be such a block).
    lisi_map, aug_map: (T, T) per-tile maps; sums: (T*T, 4) per-tile sums."""
    lisi_map = np.asarray(lisi_map, dtype=np.float64)
    aug_map = np.asarray(aug_map, dtype=np.float64)
    T = lisi_map.shape[0]
    if T % m != 0:
        raise ValueError("merge factor must divide the tile count per row")
    sums = np.asarray(sums, dtype=np.float64).reshape(T, T, 4)
    M = T // m
    out_l = np.zeros((M, M))
    out_a = np.zeros((M, M))
    for R in range(M):
        for Cc in range(M):
            blk = (slice(R * m, R * m + m), slice(Cc * m, Cc * m + m))
            out_l[R, Cc], out_a[R, Cc] = whole_from_tiles(
                lisi_map[blk], aug_map[blk], sums[blk][..., 2], sums[blk][..., 3],
                C2, C)
    return out_l, out_a
