"""Shared helpers for the GPU parity tests: run the CUDA path through the C-ABI
binding and compare it with the FP64 oracle.

Tolerance (FP32 accumulation on the GPU against the FP64 oracle): every
per-tile quantity within 1e-5 relative.
* lisi: |g - o| <= 1e-5 |o|; an oracle 0 must come back exactly 0.
* aug:  |g - o| <= 1e-5 max(|o|, r), r = B / (Sx + Sy + C) = 1 - aug.  On radio
  skies the pixels are << 1, so aug is close to 1 and a test on aug alone would
  be weak; r is checked to 1e-5 relative through the exported sums as well.
* sums A, B, Sx, Sy: each within 1e-5 relative; all terms are nonnegative, so
  the sums are perfectly conditioned; an oracle 0 must come back exactly 0.
The bound follows from the arithmetic: each per-pixel term carries a few
float32 roundings (<= ~4 u plus ~2 ulp for the approximate reciprocal,
u = 2^-24); a thread keeps two packed running sums per quantity (even and odd
elements) over one pass of at most 8 vectors, i.e. <= 32 terms each, added in
order (<= 31 u), folds the pair (1 u) and Kahan-adds the pass into its total
(~2 u); the cross-thread shuffle trees and the cluster combine add <= ~16
float32 additions.  The worst case is about 55 u = 3.3e-6, inside 1e-5.  The
per-tile ratios are IEEE float divisions of the sums (<= 3 u more); where
augLISI cancels (|aug| < r/16) it is formed in FP64 and rounded once.
"""
import numpy as np

REL = 1e-5


def to_device(a):
    import torch
    if a.dtype == np.uint16:  # bf16 bit patterns
        return torch.from_numpy(a.view(np.int16)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def widen(a):
    """Storage array -> exactly equal float32 values (the oracle's input)."""
    if a.dtype == np.uint16:
        return (a.astype(np.uint32) << 16).view(np.float32)
    return a.astype(np.float32)


def dtype_code(a):
    from paper_2501_10653_gb300 import iqa
    if a.dtype == np.float32:
        return iqa.IQA_F32
    if a.dtype == np.float16:
        return iqa.IQA_F16
    if a.dtype == np.uint16:
        return iqa.IQA_BF16
    raise TypeError(a.dtype)


def gpu_maps(ctx, x, y, NT, params=None, which="both", dx=None, dy=None):
    """Run the CUDA path; returns (lisi, aug, sums) as numpy (None where not
    requested).  dx/dy: device tensors to use instead of uploading x/y."""
    import torch
    from paper_2501_10653_gb300 import iqa
    N = x.shape[0]
    T = N // NT
    dx = to_device(x) if dx is None else dx
    dy = to_device(y) if dy is None else dy
    lisi = torch.full((T, T), float("nan"), device="cuda", dtype=torch.float32)
    aug = torch.full((T, T), float("nan"), device="cuda", dtype=torch.float32)
    sums = torch.full((T * T, 4), float("nan"), device="cuda", dtype=torch.float64)
    st = torch.cuda.current_stream()
    code = dtype_code(x)
    if which == "both":
        iqa.iqa_both(ctx, dx, dy, code, N, NT, params, lisi, aug, sums, st)
    elif which == "lisi":
        iqa.iqa_lisi(ctx, dx, dy, code, N, NT, params, lisi, None, st)
    elif which == "aug":
        iqa.iqa_auglisi(ctx, dx, dy, code, N, NT, params, aug, None, st)
    elif which == "both_nosums":
        iqa.iqa_both(ctx, dx, dy, code, N, NT, params, lisi, aug, None, st)
    torch.cuda.synchronize()
    out_l = lisi.cpu().numpy() if which in ("both", "lisi", "both_nosums") else None
    out_a = aug.cpu().numpy() if which in ("both", "aug", "both_nosums") else None
    out_s = sums.cpu().numpy() if which == "both" else None
    return out_l, out_a, out_s


def oracle_maps(orc, x, y, NT, params):
    p = params or {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}
    D = p["D"] if p.get("D", 0.0) > 0 else p["C1"] / 2
    return orc.maps(widen(x), widen(y), NT, p["C1"], p["C2"], p["C"], D, threads=8)


def assert_lisi_close(g, o, rel=REL, what="lisi"):
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    assert g.shape == o.shape
    assert np.all(np.isfinite(g)), "%s: non-finite GPU values" % what
    zero = o == 0
    assert np.all(g[zero] == 0), "%s: oracle 0 not exactly 0 on GPU" % what
    err = np.abs(g - o)
    bad = err > rel * np.abs(o)
    assert not bad.any(), "%s: %d tiles off, worst rel %.3g at %d" % (
        what, bad.sum(), np.max(err[~zero] / np.abs(o[~zero])) if (~zero).any() else 0,
        int(np.argmax(err)))


def assert_aug_close(g, o, r, rel=REL, what="aug"):
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    r = np.asarray(r, np.float64).ravel()
    assert np.all(np.isfinite(g)), "%s: non-finite GPU values" % what
    scale = np.maximum(np.abs(o), np.abs(r))
    err = np.abs(g - o)
    bad = err > rel * scale
    assert not bad.any(), "%s: %d tiles off, worst %.3g" % (
        what, bad.sum(), np.max(err / np.where(scale > 0, scale, 1)))


def assert_sums_close(g, o, rel=REL):
    g = np.asarray(g, np.float64).reshape(-1, 4)
    o = np.asarray(o, np.float64).reshape(-1, 4)
    for k, name in enumerate(("A", "B", "Sx", "Sy")):
        assert_lisi_close(g[:, k], o[:, k], rel, "sum " + name)


def assert_parity(got, want, params=None, rel=REL):
    """got/want: (lisi, aug, sums) from gpu_maps / oracle_maps."""
    gl, ga, gs = got
    ol, oa, osums = want
    p = params or {"C": 1e-6}
    r = osums[:, 1] / (osums[:, 2] + osums[:, 3] + p["C"])
    if gl is not None:
        assert_lisi_close(gl, ol, rel)
    if ga is not None:
        assert_aug_close(ga, oa, r, rel)
    if gs is not None:
        assert_sums_close(gs, osums, rel)
        gr = gs[:, 1] / (gs[:, 2] + gs[:, 3] + p["C"])
        assert_lisi_close(gr, r, rel, "r = 1 - aug")


def oracle_tile(orc, xw, yw, params=None):
    """The oracle on one N_T x N_T tile given as its two pixel windows:
    (lisi, aug, sums[4], r)."""
    p = params or {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}
    NT = xw.shape[0]
    ol, oa, os_ = oracle_maps(orc, np.ascontiguousarray(xw), np.ascontiguousarray(yw), NT, p)
    s = os_[0]
    return float(ol.ravel()[0]), float(oa.ravel()[0]), s, s[1] / (s[2] + s[3] + p["C"])


def assert_sampled(got_lisi, got_aug, picks, want, params=None, rel=REL):
    """got_*: full GPU maps (flat); picks: tile indices; want: oracle_tile()
    results for those tiles, in the same order."""
    gl = np.asarray(got_lisi).ravel()[picks]
    ga = np.asarray(got_aug).ravel()[picks]
    ol = np.array([w[0] for w in want])
    oa = np.array([w[1] for w in want])
    r = np.array([w[3] for w in want])
    assert_lisi_close(gl, ol, rel)
    assert_aug_close(ga, oa, r, rel)
