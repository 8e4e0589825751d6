"""Seeded synthetic radio-sky image pairs (input generator only).

The paper evaluates on OSKAR-simulated GLEAM skies restored with Hogbom CLEAN
(Section 3): a first epoch with 33 sources, and a second epoch with the 5
faintest removed, at N = 2048, N_T = 64.  Those images are not available, so
these generators stand in for them with the same shape: Gaussian-beam point
sources (and, for the precision workload, extended Gaussian blobs) over
Gaussian noise, a second epoch that drops the faintest sources and draws fresh
noise, and an optional faint diffuse ripple common to both epochs.

This module holds none of the method's arithmetic (no clamp, no sums, no
ratios).  Both the CUDA path's tests and the oracle's tests take their inputs
from here.

Conventions
-----------
* Beam: FWHM F gives sigma_b = F / (2 sqrt(2 ln 2)); a source of flux f at a
  continuous position is rendered as f * exp(-r^2 / (2 sigma^2)) (peak f,
  Jy/beam), evaluated within +-6 sigma.
* Noise: iid N(0, sigma^2) per pixel, an independent stream per epoch, so about
  half of the noise pixels are negative and the clamp is exercised.
* Seeds: ``np.random.default_rng([seed, stream, pair_index])`` with stream 0 =
  sky, 1 = noise of epoch 1 (x), 2 = noise of epoch 2 (y).
* Images are computed in FP64 and cast to the storage dtype at the end.
"""
import math

import numpy as np

FWHM_TO_SIGMA = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def catalog(rng, N, n_src, flux_lo, flux_hi, fwhm, ext_frac=0.0,
            ext_sigma=(5.0, 40.0)):
    """Source list: positions uniform over the image, flux log-uniform in
    [flux_lo, flux_hi]; a fraction ``ext_frac`` of sources are extended blobs
    with sigma uniform in ``ext_sigma`` pixels, the rest beam-sized."""
    px = rng.uniform(0.0, N, n_src)
    py = rng.uniform(0.0, N, n_src)
    flux = np.exp(rng.uniform(math.log(flux_lo), math.log(flux_hi), n_src))
    sigma = np.full(n_src, fwhm * FWHM_TO_SIGMA)
    if ext_frac > 0.0:
        n_ext = int(round(ext_frac * n_src))
        ext = rng.permutation(n_src)[:n_ext]
        sigma[ext] = rng.uniform(ext_sigma[0], ext_sigma[1], n_ext)
    return {"x": px, "y": py, "flux": flux, "sigma": sigma}


def drop_faintest(cat, k):
    """Second-epoch catalogue: the k lowest-flux sources removed (Section 3)."""
    keep = np.argsort(cat["flux"], kind="stable")[k:]
    keep.sort()
    return {key: v[keep] for key, v in cat.items()}


def render(cat, N):
    """FP64 N x N image of the catalogue's Gaussian sources (row = y)."""
    img = np.zeros((N, N), dtype=np.float64)
    for sx, sy, f, s in zip(cat["x"], cat["y"], cat["flux"], cat["sigma"]):
        h = int(math.ceil(6.0 * s))
        i0, i1 = max(0, int(sy) - h), min(N, int(sy) + h + 1)
        j0, j1 = max(0, int(sx) - h), min(N, int(sx) + h + 1)
        if i0 >= i1 or j0 >= j1:
            continue
        ii = np.arange(i0, i1, dtype=np.float64)[:, None] - sy
        jj = np.arange(j0, j1, dtype=np.float64)[None, :] - sx
        img[i0:i1, j0:j1] += f * np.exp(-(ii * ii + jj * jj) / (2.0 * s * s))
    return img


def ripple(rng, N, amp):
    """Faint diffuse background: three sinusoids with integer wave numbers 1-4
    along each axis and random phases, scaled so that the peak is ``amp``."""
    i = np.arange(N, dtype=np.float64)[:, None]
    j = np.arange(N, dtype=np.float64)[None, :]
    r = np.zeros((N, N))
    for _ in range(3):
        kx, ky = rng.integers(1, 5, 2)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        r += np.sin(2.0 * math.pi * (kx * j + ky * i) / N + ph)
    return r * (amp / np.max(np.abs(r)))


def _cast(img, dtype):
    if dtype in ("f32", np.float32):
        return img.astype(np.float32)
    if dtype in ("f16", np.float16):
        return img.astype(np.float16)
    if dtype == "bf16":
        # round-to-nearest-even FP64 -> FP32 -> BF16 bit pattern, as uint16
        f = img.astype(np.float32).view(np.uint32).astype(np.uint64)
        rounded = (f + 0x7FFF + ((f >> 16) & 1)) >> 16
        nan = np.isnan(img)
        out = rounded.astype(np.uint16)
        out[nan] = 0x7FC0
        return out
    raise ValueError("unknown dtype %r" % (dtype,))


def sky_pair(N, *, n_src, flux=(0.005, 2.0), fwhm=4.0, noise=2e-4, n_drop=5,
             ripple_amp=0.0, ext_frac=0.0, ext_sigma=(5.0, 40.0), seed=1,
             pair_index=0, dtype="f32"):
    """One (epoch 1, epoch 2) pair.  Epoch 2 drops the ``n_drop`` faintest
    sources and draws fresh noise; the ripple is shared.  Returns (x, y) in the
    storage dtype ("f32", "f16", or "bf16" as raw uint16 bit patterns)."""
    rng_sky = np.random.default_rng([seed, 0, pair_index])
    cat1 = catalog(rng_sky, N, n_src, flux[0], flux[1], fwhm, ext_frac, ext_sigma)
    cat2 = drop_faintest(cat1, n_drop)
    base = ripple(rng_sky, N, ripple_amp) if ripple_amp > 0 else 0.0
    x = render(cat1, N) + base
    y = render(cat2, N) + base
    x += noise * np.random.default_rng([seed, 1, pair_index]).standard_normal((N, N))
    y += noise * np.random.default_rng([seed, 2, pair_index]).standard_normal((N, N))
    return _cast(x, dtype), _cast(y, dtype)


# --- the paper-shaped workloads -------------------------------------------

#: Small single pair: N=256, N_T=64, 10 sources (FWHM 3 px, flux log-uniform
#: in [0.01, 1]), sigma 1e-3, the 3 faintest dropped, seed 0.
SMALL_PAIR_N256 = dict(N=256, NT=64, n_src=10, flux=(0.01, 1.0), fwhm=3.0,
                       noise=1e-3, n_drop=3, seed=0)

#: Paper-scale pair (Section 3): N=2048, 33 sources (FWHM 4 px, flux
#: log-uniform in [0.005, 2]), sigma 2e-4, diffuse ripple 1e-4, the 5 faintest
#: dropped, seed 1.  N_T is swept over {16, 32, 64, 128, 256}; 64 is the paper's.
PAPER_PAIR_N2048 = dict(N=2048, NT=64, n_src=33, flux=(0.005, 2.0), fwhm=4.0,
                        noise=2e-4, n_drop=5, ripple_amp=1e-4, seed=1)
PAPER_NT_SWEEP = (16, 32, 64, 128, 256)


def small_pair(dtype="f32"):
    w = dict(SMALL_PAIR_N256)
    w.pop("NT")
    return sky_pair(dtype=dtype, **w)


def paper_pair(pair_index=0, dtype="f32", N=None):
    w = dict(PAPER_PAIR_N2048)
    w.pop("NT")
    if N is not None:
        w["n_src"] = max(1, int(round(33 * (N / 2048.0) ** 2)))
        w["n_drop"] = max(1, int(math.ceil(0.1 * w["n_src"]))) if N != 2048 else 5
        w["N"] = N
    return sky_pair(pair_index=pair_index, dtype=dtype, **w)


def paper_pair_dropped(pair_index=0):
    """The sources that epoch 2 of ``paper_pair(pair_index)`` leaves out: the
    same catalogue draw (the sky stream's first draw), its ``n_drop``
    faintest.  Returns their (x, y, flux) arrays, columns x and rows y in
    pixels."""
    w = dict(PAPER_PAIR_N2048)
    rng_sky = np.random.default_rng([w["seed"], 0, pair_index])
    cat = catalog(rng_sky, w["N"], w["n_src"], w["flux"][0], w["flux"][1], w["fwhm"])
    gone = np.argsort(cat["flux"], kind="stable")[:w["n_drop"]]
    return cat["x"][gone], cat["y"][gone], cat["flux"][gone]


def mixed_batch_specs(n_pairs=64, seed=2):
    """The batched workload's draw: N from {1024, 2048, 4096, 8192} with weights
    4:3:2:1 and N_T from {32, 64, 128}, per pair.  Returns a list of (N, NT)."""
    rng = np.random.default_rng([seed, 3])
    Ns = rng.choice([1024, 2048, 4096, 8192], size=n_pairs,
                    p=np.array([4, 3, 2, 1]) / 10.0)
    NTs = rng.choice([32, 64, 128], size=n_pairs)
    return [(int(a), int(b)) for a, b in zip(Ns, NTs)]


def mixed_batch_pair(i, N, seed=2, dtype="f32"):
    """Pair i of the batched workload: the paper-scale sky scaled to N, with
    round(33 (N/2048)^2) sources and ceil(10%) of them dropped in epoch 2."""
    n_src = max(1, int(round(33 * (N / 2048.0) ** 2)))
    return sky_pair(N, n_src=n_src, flux=(0.005, 2.0), fwhm=4.0, noise=2e-4,
                    n_drop=int(math.ceil(0.1 * n_src)), ripple_amp=1e-4,
                    seed=seed, pair_index=i, dtype=dtype)


def precision_pair(i, N=8192, seed=3, dtype="f32"):
    """Pair i of the precision workload: 33 sources per pair, half point
    sources (FWHM 4) and half extended blobs (sigma 5-40 px), peak flux
    log-uniform in [1e-4, 1] (1e4 dynamic range), sigma 5e-3 noise, epoch 2
    drops the faintest 10%.  Returns FP64-derived images in ``dtype``."""
    return sky_pair(N, n_src=33, flux=(1e-4, 1.0), fwhm=4.0, noise=5e-3,
                    n_drop=4, ext_frac=0.5, seed=seed, pair_index=i, dtype=dtype)


# --- device-reproducible epochs (the serving workload) -----------------------
#
# The serving loop renders epochs on the device (csrc/iqa_synth.cu).  The
# functions below make the same images on the host, bit for bit, so that tests
# can feed the oracle inputs that never came from the CUDA path:
#   * noise: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11), key = seed,
#     counter = (q low word, q high word, 0x5EED, 0) with q = pixel index / 4;
#     word k serves pixel 4q + k: the sum s of its four bytes gives
#     z = (s - 510) * (sqrt(3) / 256) in float32 (Irwin-Hall of four uniforms
#     on the byte centres: zero mean, variance 1 - 2^-16, bounded at
#     +-sqrt(12));
#   * sources: integer centres, float32 1-D profiles g[-h..h]; contribution
#     (f * g[dy]) * g[dx], added to the pixel in catalogue order;
#   * pixel = sky + sigma * z in float32, rounded to nearest into storage.

_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over uint32 counter arrays; returns 4 words."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3))
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0)), lo1, (hi0 ^ c3 ^ np.uint64(k1)), lo0
        k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def epoch_noise(N, seed):
    """float32 N x N standardised noise z of the device generator: one Philox
    call per four horizontally adjacent pixels (q = pixel index / 4), word k
    for pixel 4q + k, z = (byte sum - 510) * (sqrt(3) / 256)."""
    q = np.arange(N * N // 4, dtype=np.uint64)
    w = philox4x32_10(q & _MASK32, q >> np.uint64(32), np.uint64(0x5EED),
                      np.uint64(0), seed & 0xFFFFFFFF, seed >> 32)
    scale = np.float32(1.7320508075688772) / np.float32(256.0)
    z = np.empty(N * N, dtype=np.float32)
    for k in range(4):
        b = w[k].astype(np.uint32).view(np.uint8).reshape(-1, 4).astype(np.int32)
        z[k::4] = (b.sum(axis=1) - 510).astype(np.float32) * scale
    return z.reshape(N, N)


def serving_catalog(N, ref_index, seed=4, fwhm=4.0, flux=(0.005, 2.0), noise=2e-4):
    """A reference sky of the serving workload: round(33 (N/2048)^2) Gaussian-beam
    sources at integer centres, flux log-uniform, with float32 profiles."""
    rng = np.random.default_rng([seed, 5, ref_index])
    n_src = max(1, int(round(33 * (N / 2048.0) ** 2)))
    sig = fwhm * FWHM_TO_SIGMA
    h = int(math.ceil(6.0 * sig))
    k = np.arange(-h, h + 1, dtype=np.float64)
    prof = np.exp(-(k * k) / (2.0 * sig * sig)).astype(np.float32)
    return {
        "N": N,
        "x": rng.integers(0, N, n_src).astype(np.int32),
        "y": rng.integers(0, N, n_src).astype(np.int32),
        "flux": np.exp(rng.uniform(math.log(flux[0]), math.log(flux[1]), n_src)
                       ).astype(np.float32),
        "half": np.full(n_src, h, dtype=np.int32),
        "profile_off": (np.arange(n_src, dtype=np.int32) * (2 * h + 1)),
        "profile": np.tile(prof, n_src),
        "noise_sigma": np.float32(noise),
    }


def _noise_window(N, seed, r0, r1, c0, c1):
    """epoch_noise(N, seed)[r0:r1, c0:c1], computed for those pixels only
    (pixel p = r N + c takes word p % 4 of the Philox call for p / 4)."""
    rows = np.arange(r0, r1, dtype=np.uint64)[:, None]
    cols = np.arange(c0, c1, dtype=np.uint64)[None, :]
    p = rows * np.uint64(N) + cols
    q = p >> np.uint64(2)
    w = philox4x32_10(q & _MASK32, q >> np.uint64(32), np.uint64(0x5EED), np.uint64(0),
                      seed & 0xFFFFFFFF, seed >> 32)
    word = np.choose((p & np.uint64(3)).astype(np.int64), w)
    b = sum((word >> np.uint64(8 * k)) & np.uint64(0xFF) for k in range(4)).astype(np.int64)
    scale = np.float32(1.7320508075688772) / np.float32(256.0)
    return (b - 510).astype(np.float32) * scale


def render_epoch_window(cat, seed, r0, r1, c0, c1, drop=(), add=None, dtype="f32"):
    """render_epoch(cat, seed, drop, add, dtype)[r0:r1, c0:c1], computed for
    that window only (the same float32 operations, pixel by pixel)."""
    N = cat["N"]
    sky = np.zeros((r1 - r0, c1 - c0), dtype=np.float32)
    drop = set(int(d) for d in drop)

    def put(i, cx, cy, f):
        h = int(cat["half"][i])
        g = cat["profile"][cat["profile_off"][i]:cat["profile_off"][i] + 2 * h + 1]
        a0, a1 = max(r0, cy - h), min(r1, cy + h + 1)
        b0, b1 = max(c0, cx - h), min(c1, cx + h + 1)
        if a0 >= a1 or b0 >= b1:
            return
        gy = np.float32(f) * g[a0 - cy + h:a1 - cy + h]
        gx = g[b0 - cx + h:b1 - cx + h]
        sky[a0 - r0:a1 - r0, b0 - c0:b1 - c0] = (sky[a0 - r0:a1 - r0, b0 - c0:b1 - c0]
                                                 + gy[:, None] * gx[None, :])

    for i in range(len(cat["x"])):
        if i in drop:
            continue
        put(i, int(cat["x"][i]), int(cat["y"][i]), cat["flux"][i])
    if add is not None:
        put(int(add[0]), int(add[1]), int(add[2]), np.float32(add[3]))
    if (r0, r1, c0, c1) == (0, N, 0, N):
        z = epoch_noise(N, seed)
    else:
        z = _noise_window(N, seed, r0, r1, c0, c1)
    img = sky + np.float32(cat["noise_sigma"]) * z
    return _cast(img.astype(np.float32), dtype) if dtype != "f32" else img


def render_epoch(cat, seed, drop=(), add=None, dtype="f32"):
    """Host mirror of the device epoch generator.  add = (src, x, y, flux) puts
    a transient with source `src`'s profile at (x, y)."""
    N = cat["N"]
    return render_epoch_window(cat, seed, 0, N, 0, N, drop, add, dtype)


def catalog_without_faintest(cat, k):
    """A serving catalogue with its k lowest-flux sources removed (the second
    epoch of the batched workload); profiles stay shared."""
    keep = np.sort(np.argsort(cat["flux"], kind="stable")[k:])
    out = dict(cat)
    for key in ("x", "y", "flux", "half", "profile_off"):
        out[key] = cat[key][keep]
    return out
