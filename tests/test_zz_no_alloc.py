"""iqa_batch_noalloc, the batched launch for callers that cannot allocate device
memory (a pipeline that reserves all GPU memory at start-up, or that cannot
afford an allocation's device-wide synchronisation mid-run), against the
existing one-pair entry point iqa_both, through the C-ABI (needs a GPU).

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before it; it also passes on its own in a
fresh process.
"""
import numpy as np
import pytest

import parity
from paper_2501_10653_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}


@pytest.fixture(scope="module")
def lib_ctx():
    from paper_2501_10653_gb300 import build, iqa
    build.build()
    h = iqa.iqa_create(0, 0)
    yield h
    iqa.iqa_destroy(h)


def _batch(specs, seed, dtype="f32"):
    import torch
    items = []
    for i, (N, NT) in enumerate(specs):
        x, y = synth.mixed_batch_pair(i, N, seed=seed, dtype=dtype)
        T = N // NT
        items.append(dict(N=N, NT=NT, x=x, y=y, code=parity.dtype_code(x),
                          dx=parity.to_device(x), dy=parity.to_device(y),
                          l=torch.full((T * T,), float("nan"), device="cuda"),
                          a=torch.full((T * T,), float("nan"), device="cuda"),
                          s=torch.full((T * T, 4), float("nan"), device="cuda",
                                       dtype=torch.float64)))
    return items


def _reference(ctx, it):
    """The same pair through the existing entry point iqa_both."""
    import torch
    from paper_2501_10653_gb300 import iqa
    T = it["N"] // it["NT"]
    l = torch.empty(T * T, device="cuda")
    a = torch.empty(T * T, device="cuda")
    s = torch.empty((T * T, 4), device="cuda", dtype=torch.float64)
    iqa.iqa_both(ctx, it["dx"], it["dy"], it["code"], it["N"], it["NT"], PARAMS, l, a, s,
                 torch.cuda.current_stream())
    torch.cuda.synchronize()
    return l.cpu().numpy(), a.cpu().numpy(), s.cpu().numpy()


def _check_against_reference(ctx, items, orc=None):
    """Every pair's maps and sums against iqa_both on the same pair, and, when
    the oracle is given, against the FP64 oracle on the same stored pixels."""
    for it in items:
        want = _reference(ctx, it)
        got = (it["l"].cpu().numpy(), it["a"].cpu().numpy(), it["s"].cpu().numpy())
        parity.assert_parity(got, want, PARAMS)
        if orc is not None:
            ol, oa, osums = parity.oracle_maps(orc, it["x"], it["y"], it["NT"], PARAMS)
            parity.assert_parity(got, (ol.ravel(), oa.ravel(), osums), PARAMS)


def _pairs(items):
    from paper_2501_10653_gb300 import iqa
    return [iqa.make_pair(it["dx"], it["dy"], it["N"], it["NT"], it["l"], it["a"], it["s"])
            for it in items]


def test_noalloc_matches_existing_entry_point_on_two_calls_in_a_row(lib_ctx, orc):
    import torch
    from paper_2501_10653_gb300 import iqa
    st = torch.cuda.current_stream()
    first = _batch([(1024, 64), (512, 32), (256, 128), (768, 96)], seed=21)
    second = _batch([(512, 128), (1024, 32), (256, 64)], seed=22)
    pairs1 = [iqa.make_pair(it["dx"], it["dy"], it["N"], it["NT"], it["l"], it["a"], it["s"])
              for it in first]
    pairs2 = [iqa.make_pair(it["dx"], it["dy"], it["N"], it["NT"], it["l"], it["a"], it["s"])
              for it in second]
    iqa.iqa_batch_noalloc(pairs1, iqa.IQA_F32, PARAMS, st)
    iqa.iqa_batch_noalloc(pairs2, iqa.IQA_F32, PARAMS, st)
    torch.cuda.synchronize()
    _check_against_reference(lib_ctx, first, orc)
    _check_against_reference(lib_ctx, second, orc)
    # alternating calls rewrite the same array entries with other pairs: every
    # call must see its own descriptors, and the counters start at zero
    for batch, pairs in ((first, pairs1), (second, pairs2), (first, pairs1)):
        for it in batch:
            it["l"].fill_(float("nan"))
            it["a"].fill_(float("nan"))
            it["s"].fill_(float("nan"))
        iqa.iqa_batch_noalloc(pairs, iqa.IQA_F32, PARAMS, st)
        torch.cuda.synchronize()
        _check_against_reference(lib_ctx, batch)


def test_noalloc_rejects_more_pairs_than_its_array_holds(lib_ctx):
    import torch
    from paper_2501_10653_gb300 import iqa
    d = torch.zeros(256 * 256, device="cuda")
    m = torch.zeros(16, device="cuda")
    p = iqa.make_pair(d, d, 256, 64, m)
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_batch_noalloc([p] * (iqa.IQA_NOALLOC_MAX_PAIRS + 1), iqa.IQA_F32, PARAMS,
                              torch.cuda.current_stream())
    assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
    assert "at most" in iqa.iqa_last_error(None)
    torch.cuda.synchronize()
    assert np.all(m.cpu().numpy() == 0)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_noalloc_16bit_storage_two_calls(lib_ctx, orc, dt):
    """16-bit storage takes the 16-bit default shape of the persistent kernel."""
    import torch
    from paper_2501_10653_gb300 import iqa
    st = torch.cuda.current_stream()
    first = _batch([(1024, 64), (512, 128), (256, 32)], seed=23, dtype=dt)
    second = _batch([(768, 96), (512, 64)], seed=24, dtype=dt)
    code = first[0]["code"]
    iqa.iqa_batch_noalloc(_pairs(first), code, PARAMS, st)
    iqa.iqa_batch_noalloc(_pairs(second), code, PARAMS, st)
    torch.cuda.synchronize()
    _check_against_reference(lib_ctx, first, orc)
    _check_against_reference(lib_ctx, second, orc)


def test_noalloc_full_table_of_small_pairs(lib_ctx):
    """A call of exactly IQA_NOALLOC_MAX_PAIRS pairs: the whole descriptor
    table, twice in a row with the pairs in another order."""
    import torch
    from paper_2501_10653_gb300 import iqa
    rng = np.random.default_rng(31)
    specs = [(int(rng.choice([128, 256])), int(rng.choice([16, 32, 64])))
             for _ in range(iqa.IQA_NOALLOC_MAX_PAIRS)]
    items = _batch(specs, seed=25)
    st = torch.cuda.current_stream()
    iqa.iqa_batch_noalloc(_pairs(items), iqa.IQA_F32, PARAMS, st)
    torch.cuda.synchronize()
    _check_against_reference(lib_ctx, items)
    for it in items:
        it["l"].fill_(float("nan"))
        it["a"].fill_(float("nan"))
        it["s"].fill_(float("nan"))
    iqa.iqa_batch_noalloc(_pairs(items[::-1]), iqa.IQA_F32, PARAMS, st)
    torch.cuda.synchronize()
    _check_against_reference(lib_ctx, items)


def test_noalloc_rejects_misaligned_images_and_writes_nothing(lib_ctx):
    import torch
    from paper_2501_10653_gb300 import iqa
    buf = torch.zeros(256 * 256 + 4, device="cuda")
    m = torch.full((16,), float("nan"), device="cuda")
    good = iqa.make_pair(buf, buf, 256, 64, m)
    bad = iqa.make_pair(buf.data_ptr() + 4, buf, 256, 64, m)
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_batch_noalloc([good, bad], iqa.IQA_F32, PARAMS, torch.cuda.current_stream())
    assert ei.value.status == iqa.IQA_ERR_UNSUPPORTED
    assert "aligned" in iqa.iqa_last_error(None)
    torch.cuda.synchronize()
    assert np.all(np.isnan(m.cpu().numpy()))
