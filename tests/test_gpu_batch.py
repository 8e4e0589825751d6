"""Batched form (one persistent launch over many pairs), through the C-ABI
plan API, against the FP64 oracle (needs a GPU)."""
import numpy as np
import pytest

import parity
from paper_2501_10653_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}


@pytest.fixture(scope="module")
def ctx():
    from paper_2501_10653_gb300 import build, iqa
    build.build()
    h = iqa.iqa_create(0, 0)
    yield h
    iqa.iqa_destroy(h)


def _specs():
    # a small stand-in for the mixed batch: N from {256, 512, 1024}, N_T from
    # {32, 64, 128}, several tiles per unit and several chunks per unit
    return [(1024, 64), (256, 32), (512, 128), (1024, 32), (512, 64), (256, 128),
            (1024, 128), (512, 32), (256, 64), (1024, 64), (768, 96), (640, 80)]


class Batch:
    def __init__(self, specs, dtype="f32", seed=2):
        import torch
        self.specs = specs
        self.host = [synth.mixed_batch_pair(i, N, seed=seed, dtype=dtype)
                     for i, (N, _) in enumerate(specs)]
        self.dev = [(parity.to_device(x), parity.to_device(y)) for x, y in self.host]
        self.out = []
        for N, NT in specs:
            T = N // NT
            self.out.append((torch.full((T * T,), float("nan"), device="cuda"),
                             torch.full((T * T,), float("nan"), device="cuda"),
                             torch.full((T * T, 4), float("nan"), device="cuda",
                                        dtype=torch.float64)))

    def pairs(self, idx=None):
        from paper_2501_10653_gb300 import iqa
        idx = range(len(self.specs)) if idx is None else idx
        return [iqa.make_pair(self.dev[i][0], self.dev[i][1], self.specs[i][0],
                              self.specs[i][1], *self.out[i]) for i in idx]

    def results(self, i):
        return tuple(t.cpu().numpy() for t in self.out[i])


def _run(ctx, batch, idx=None, flags=1, dtype_code=0, launches=1):
    import torch
    from paper_2501_10653_gb300 import iqa
    plan = iqa.iqa_plan_create(ctx, batch.pairs(idx), dtype_code, PARAMS, flags)
    try:
        for _ in range(launches):
            iqa.iqa_plan_launch(plan, torch.cuda.current_stream())
        iqa.iqa_wait(ctx, torch.cuda.current_stream(), 20_000_000)
        info = iqa.iqa_plan_info(plan)
    finally:
        iqa.iqa_plan_destroy(plan)
    return info


def test_mixed_batch_against_oracle(ctx, orc):
    b = Batch(_specs())
    info = _run(ctx, b)
    assert info.npairs == len(b.specs) and info.graph == 1
    for i, (N, NT) in enumerate(b.specs):
        x, y = b.host[i]
        want = parity.oracle_maps(orc, x, y, NT, PARAMS)
        gl, ga, gs = b.results(i)
        parity.assert_parity((gl.reshape(N // NT, -1), ga.reshape(N // NT, -1), gs),
                             want, PARAMS)


@pytest.mark.parametrize("dt,code", [("f16", 1), ("bf16", 2)])
def test_mixed_batch_16bit(ctx, orc, dt, code):
    b = Batch(_specs()[:6], dtype=dt)
    _run(ctx, b, dtype_code=code)
    for i, (N, NT) in enumerate(b.specs):
        x, y = b.host[i]
        want = parity.oracle_maps(orc, x, y, NT, PARAMS)
        parity.assert_parity(b.results(i), want, PARAMS)


def test_same_alone_and_in_the_mix(ctx):
    """Each pair's maps are bit-identical whether it runs alone or with others."""
    b = Batch(_specs())
    _run(ctx, b)
    mixed = [b.results(i) for i in range(len(b.specs))]
    for i in (0, 3, 5, 10):
        for t in b.out[i]:
            t.fill_(float("nan"))
        _run(ctx, b, idx=[i])
        alone = b.results(i)
        for u, v in zip(alone, mixed[i]):
            assert np.array_equal(u, v), "pair %d differs alone vs in the mix" % i


def test_graph_direct_and_repeated_launches_agree(ctx):
    """Graph replay, direct launch and back-to-back launches (the work counter
    resets itself) all give the same bits."""
    b = Batch(_specs()[:8])
    _run(ctx, b, flags=0)
    direct = [b.results(i) for i in range(8)]
    _run(ctx, b, flags=1, launches=4)
    for i in range(8):
        for u, v in zip(b.results(i), direct[i]):
            assert np.array_equal(u, v)


def test_plan_autotune_keeps_parity(ctx, orc):
    import torch
    from paper_2501_10653_gb300 import iqa
    b = Batch(_specs()[:6])
    plan = iqa.iqa_plan_create(ctx, b.pairs(), 0, PARAMS, iqa.IQA_PLAN_GRAPH)
    try:
        best = iqa.iqa_plan_autotune(plan, torch.cuda.current_stream(), 2)
        assert best.variant == 1 and best.threads in (128, 256, 512)
        for t in b.out:
            for u in t:
                u.fill_(float("nan"))
        iqa.iqa_plan_launch(plan, torch.cuda.current_stream())
        iqa.iqa_wait(ctx, torch.cuda.current_stream(), 20_000_000)
    finally:
        iqa.iqa_plan_destroy(plan)
    for i, (N, NT) in enumerate(b.specs):
        x, y = b.host[i]
        parity.assert_parity(b.results(i), parity.oracle_maps(orc, x, y, NT, PARAMS),
                             PARAMS)


def test_plan_rejects_bad_pairs(ctx):
    import torch
    from paper_2501_10653_gb300 import iqa
    d = torch.zeros(256 * 256 + 4, device="cuda")
    m = torch.zeros(64, device="cuda")
    bad = [iqa.make_pair(d, None, 256, 32, m),
           iqa.make_pair(d, d, 256, 48, m),
           iqa.make_pair(d[1:], d, 256, 32, m),
           iqa.make_pair(d, d, 256, 32)]
    for p in bad:
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_plan_create(ctx, [p], 0, PARAMS)
        assert ei.value.status in (iqa.IQA_ERR_INVALID_ARG, iqa.IQA_ERR_UNSUPPORTED)


def test_device_wait_timeout_reports_and_context_recovers(ctx, orc):
    """Failure path without a GPU fault: the producer is told to issue nothing,
    so every consumer wait runs out after 20 ms; the kernel records the error
    and returns, iqa_wait reports IQA_ERR_TIMEOUT, and the next launch on the
    same context is correct."""
    import torch
    from paper_2501_10653_gb300 import iqa
    b = Batch(_specs()[:3])
    st = torch.cuda.current_stream()
    plan = iqa.iqa_plan_create(ctx, b.pairs(), 0, PARAMS, 0)
    try:
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_WAIT_TIMEOUT_US, 20_000)
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INJECT_STALL, 1)
        iqa.iqa_plan_launch(plan, st)
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_wait(ctx, st, 20_000_000)
        assert ei.value.status == iqa.IQA_ERR_TIMEOUT
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INJECT_STALL, 0)
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_WAIT_TIMEOUT_US, 1_000_000)
        iqa.iqa_plan_launch(plan, st)
        iqa.iqa_wait(ctx, st, 20_000_000)
    finally:
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INJECT_STALL, 0)
        iqa.iqa_plan_destroy(plan)
    for i, (N, NT) in enumerate(b.specs):
        x, y = b.host[i]
        parity.assert_parity(b.results(i), parity.oracle_maps(orc, x, y, NT, PARAMS),
                             PARAMS)


def test_rewritten_descriptor_tables_are_reread(ctx, orc):
    """Plans created one after another reuse the same device table addresses
    with new tensor maps; each launch must read the new maps (the kernel
    acquires every table-resident tensor map before first use)."""
    import torch
    from paper_2501_10653_gb300 import iqa
    sets = [Batch([(512, 64), (1024, 32)], seed=31), Batch([(1024, 128), (256, 16)], seed=32),
            Batch([(768, 96), (512, 32)], seed=33)]
    for rep in range(2):
        for b in sets:
            for t in b.out:
                for u in t:
                    u.fill_(float("nan"))
            _run(ctx, b, flags=rep)
            for i, (N, NT) in enumerate(b.specs):
                x, y = b.host[i]
                parity.assert_parity(b.results(i), parity.oracle_maps(orc, x, y, NT, PARAMS),
                                     PARAMS)


@pytest.mark.parametrize("dt,code", [("f32", 0), ("f16", 1), ("bf16", 2)])
def test_independent_plans_back_to_back(ctx, orc, dt, code):
    """IQA_PLAN_INDEPENDENT: each CTA copies its first unit while the kernel
    before it drains, and waits for that kernel before its shared counter.
    Eight independent plans over the same pairs, each writing its own
    NaN-filled maps, launched back to back (each launch's head overlaps the
    previous one's tail), then one plan launched six times back to back:
    every map fully written and bit-identical to a default plan's, whose
    maps match the oracle."""
    import torch
    from paper_2501_10653_gb300 import iqa
    specs = _specs()[:8]
    ref = Batch(specs, dtype=dt)
    _run(ctx, ref, flags=0, dtype_code=code)
    want = [ref.results(i) for i in range(len(specs))]
    for i, (N, NT) in enumerate(specs[:3]):
        x, y = ref.host[i]
        parity.assert_parity(want[i], parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)
    outs = [Batch.__new__(Batch) for _ in range(8)]
    plans = []
    try:
        for o in outs:
            o.specs, o.host, o.dev = ref.specs, ref.host, ref.dev
            o.out = [tuple(torch.full_like(t, float("nan")) for t in ref.out[i])
                     for i in range(len(specs))]
            plans.append(iqa.iqa_plan_create(ctx, o.pairs(), code, PARAMS,
                                             iqa.IQA_PLAN_INDEPENDENT))
        st = torch.cuda.current_stream()
        for p in plans:
            iqa.iqa_plan_launch(p, st)
        for _ in range(5):
            iqa.iqa_plan_launch(plans[0], st)
        iqa.iqa_wait(ctx, st, 20_000_000)
    finally:
        for p in plans:
            iqa.iqa_plan_destroy(p)
    for o in outs:
        for i in range(len(specs)):
            for u, v in zip(o.results(i), want[i]):
                assert np.array_equal(u, v)


def test_plan_rejects_unknown_flags(ctx):
    from paper_2501_10653_gb300 import iqa
    b = Batch(_specs()[:1])
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_plan_create(ctx, b.pairs(), iqa.IQA_F32, PARAMS, 4)
    assert ei.value.status == iqa.IQA_ERR_INVALID_ARG


@pytest.mark.parametrize("dt,code", [("f32", 0), ("f16", 1)])
def test_small_unit_plans_static_first_grab(ctx, orc, dt, code):
    """Plans of N_T = 16 pairs, whose units (several tile rows of at most 32
    tiles) hold 32-64 KB of each image: each CTA's static first grab then spans
    several units, and dynamic grabs count from the grid size times that.  Independent plans
    back to back into NaN-filled maps, and a one-pair plan with fewer units
    than the grid's first grabs: every map written, bit-identical to a
    stream-ordered plan, which matches the oracle."""
    import torch
    from paper_2501_10653_gb300 import iqa
    specs = [(512, 16), (1024, 16), (256, 16), (768, 16)]
    ref = Batch(specs, dtype=dt, seed=41)
    _run(ctx, ref, flags=0, dtype_code=code)
    want = [ref.results(i) for i in range(len(specs))]
    for i, (N, NT) in enumerate(specs):
        x, y = ref.host[i]
        parity.assert_parity(want[i], parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)
    outs = [Batch.__new__(Batch) for _ in range(4)]
    plans = []
    try:
        for o in outs:
            o.specs, o.host, o.dev = ref.specs, ref.host, ref.dev
            o.out = [tuple(torch.full_like(t, float("nan")) for t in ref.out[i])
                     for i in range(len(specs))]
            plans.append(iqa.iqa_plan_create(ctx, o.pairs(), code, PARAMS,
                                             iqa.IQA_PLAN_INDEPENDENT))
        st = torch.cuda.current_stream()
        for _ in range(3):
            for p in plans:
                iqa.iqa_plan_launch(p, st)
        iqa.iqa_wait(ctx, st, 20_000_000)
    finally:
        for p in plans:
            iqa.iqa_plan_destroy(p)
    for o in outs:
        for i in range(len(specs)):
            for u, v in zip(o.results(i), want[i]):
                assert np.array_equal(u, v)
    # one N=256 pair: a few units, fewer than the grid's first grabs
    one = Batch([(256, 16)], dtype=dt, seed=42)
    _run(ctx, one, flags=iqa.IQA_PLAN_INDEPENDENT, dtype_code=code, launches=3)
    x, y = one.host[0]
    parity.assert_parity(one.results(0), parity.oracle_maps(orc, x, y, 16, PARAMS), PARAMS)


def _plan_with_shape(ctx, batch, shape, flags=0, dtype_code=0, launches=1):
    import torch
    from paper_2501_10653_gb300 import iqa
    plan = iqa.iqa_plan_create(ctx, batch.pairs(), dtype_code, PARAMS, flags)
    try:
        iqa.iqa_plan_set_config(plan, shape)
        for t in batch.out:
            for u in t:
                u.fill_(float("nan"))
        for _ in range(launches):
            iqa.iqa_plan_launch(plan, torch.cuda.current_stream())
        iqa.iqa_wait(ctx, torch.cuda.current_stream(), 20_000_000)
        info = iqa.iqa_plan_info(plan)
    finally:
        iqa.iqa_plan_destroy(plan)
    return info


# (N, N_T, storage, threads, unit_kpx, tiles across TX, tile rows per unit RH):
# a unit of RH > 1 tile rows keeps per-tile-row partials (up to twice the
# consumer threads of reduction slots) and reduces them at its end.  Cases: RH
# 1 / 2 / 4 (128-vector unit rows); RH 18 on 8-vector unit rows (a warp spans
# four unit rows; 144 slots, more than the 128 threads); 3-D boxes
# (1024-element unit rows); 16-bit storage (RH 4 with 256 slots).
MULTI_ROW = [
    (1024, 16, "f32", 128, 8, 32, 1),
    (1024, 16, "f32", 128, 16, 32, 2),
    (1024, 16, "f32", 128, 32, 32, 4),
    (288, 16, "f32", 128, 32, 2, 18),
    (2048, 32, "f32", 256, 64, 32, 2),
    (768, 16, "f16", 128, 32, 16, 4),
    (1024, 16, "f16", 128, 128, 64, 4),
    (512, 8, "f32", 128, 64, 64, 4),
]


@pytest.mark.parametrize("N,NT,dt,threads,kpx,TX,RH", MULTI_ROW)
def test_multi_row_units_against_oracle(ctx, orc, N, NT, dt, threads, kpx, TX, RH):
    """Units of several tile rows: the plan's work list has (N/NT/RH) *
    (N/NT/TX) units, and every tile (maps and exported sums) matches the
    oracle."""
    b = Batch([(N, NT)], dtype=dt, seed=51)
    code = {"f32": 0, "f16": 1, "bf16": 2}[dt]
    info = _plan_with_shape(ctx, b, {"threads": threads, "unit_kpx": kpx}, dtype_code=code)
    T = N // NT
    assert info.total_units == (T // RH) * (T // TX)
    assert info.config.unit_kpx == kpx and info.config.threads == threads
    x, y = b.host[0]
    parity.assert_parity(b.results(0), parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)


def test_multi_row_units_change_no_bit(ctx):
    """At the same unit width a thread sums the same columns of the same chunks
    whatever the tile rows per unit, so 1, 2, 4 and 8 rows (256 reduction
    slots) give the same bits, stream-ordered and as independent launches back
    to back."""
    from paper_2501_10653_gb300 import iqa
    b = Batch([(1024, 16), (512, 16)], seed=52)
    _plan_with_shape(ctx, b, {"unit_kpx": 8})
    want = [b.results(i) for i in range(2)]
    for kpx in (16, 32, 64):
        for flags, launches in ((0, 1), (iqa.IQA_PLAN_INDEPENDENT | iqa.IQA_PLAN_GRAPH, 3)):
            _plan_with_shape(ctx, b, {"unit_kpx": kpx}, flags=flags, launches=launches)
            for i in range(2):
                for u, v in zip(b.results(i), want[i]):
                    assert np.array_equal(u, v), (kpx, flags, i)


def test_plan_set_config_rejects_and_keeps_shape(ctx):
    import torch
    from paper_2501_10653_gb300 import iqa
    b = Batch([(512, 16)], seed=53)
    plan = iqa.iqa_plan_create(ctx, b.pairs(), 0, PARAMS, iqa.IQA_PLAN_GRAPH)
    try:
        iqa.iqa_plan_set_config(plan, {"unit_kpx": 16})
        before = iqa.iqa_plan_info(plan)
        for bad in ({"unit_kpx": 0}, {"unit_kpx": 2048}, {"variant": 0},
                    {"stages": 1}, {"threads": 96}, {"stage_kb": 32},
                    {"stages": 16, "stage_kb": 16}):
            with pytest.raises(iqa.IqaError) as ei:
                iqa.iqa_plan_set_config(plan, bad)
            assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
            after = iqa.iqa_plan_info(plan)
            assert (after.total_units, after.config.unit_kpx, after.config.stages,
                    after.config.threads) == (before.total_units, before.config.unit_kpx,
                                              before.config.stages, before.config.threads)
        iqa.iqa_plan_launch(plan, torch.cuda.current_stream())
        iqa.iqa_wait(ctx, torch.cuda.current_stream(), 20_000_000)
    finally:
        iqa.iqa_plan_destroy(plan)
    assert np.all(np.isfinite(b.results(0)[0]))
