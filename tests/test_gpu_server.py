"""Serving loop on the GPU, through the C-ABI (needs a GPU).

The second epochs are rendered on the device; the host mirror of the generator
(synth.render_epoch) makes the same images bit for bit, so the oracle runs on
inputs that did not come from the CUDA path."""
import time

import numpy as np
import pytest

import parity
from paper_2501_10653_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}
REFS = ((0, 512), (1, 1024), (2, 2048))


@pytest.fixture(scope="module")
def ctx():
    from paper_2501_10653_gb300 import build, iqa
    build.build()
    h = iqa.iqa_create(0, 0)
    yield h
    iqa.iqa_destroy(h)


def _server(ctx, dtype, **kw):
    from paper_2501_10653_gb300 import iqa
    args = dict(dtype=dtype, max_pairs_per_step=8, max_inflight_steps=2,
                pool_bytes=512 << 20, params=PARAMS)
    args.update(kw)
    srv = iqa.iqa_server_create(ctx, **args)
    cats = {}
    for rid, N in REFS:
        cats[rid] = synth.serving_catalog(N, rid)
        iqa.iqa_server_add_reference(srv, rid, cats[rid], 500 + rid)
    return srv, cats


def _wait(iqa, srv, hs, timeout_s=60.0):
    t0 = time.time()
    for h in hs:
        while iqa.iqa_poll(srv, h, 200_000) == iqa.IQA_PENDING:
            assert time.time() - t0 < timeout_s


def _result(iqa, srv, h, T):
    l = np.full(T * T, np.nan, np.float32)
    a = np.full(T * T, np.nan, np.float32)
    iqa.iqa_result(srv, h, l, a)
    return l, a


DT = {"f32": 0, "f16": 1, "bf16": 2}


@pytest.mark.parametrize("dt", ["f16", "f32", "bf16"])
def test_device_references_match_host_mirror_bitwise(ctx, dt):
    from paper_2501_10653_gb300 import iqa
    srv, cats = _server(ctx, DT[dt])
    try:
        for rid, N in REFS:
            want = synth.render_epoch(cats[rid], 500 + rid, dtype=dt)
            got = np.empty_like(want)
            iqa.iqa_server_reference_image(srv, rid, got)
            assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (dt, rid)
    finally:
        iqa.iqa_server_destroy(srv)


def test_served_maps_against_oracle(ctx, orc):
    """Requests of mixed N and N_T, with drops and a transient, served in
    batched steps: each map against the oracle on host-mirrored inputs."""
    from paper_2501_10653_gb300 import iqa
    srv, cats = _server(ctx, iqa.IQA_F16, time_kernels=1)
    reqs = [(0, 32, 11, [0], None), (1, 64, 12, [1, 3], (2, 700, 300, 0.8)),
            (2, 128, 13, [4, 5, 6], None), (2, 64, 14, [], (0, 1500, 99, 0.05)),
            (1, 32, 15, [2], None), (0, 128, 16, [1], (1, 20, 400, 1.5))]
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(r, nt, sd, dr, ad))
              for r, nt, sd, dr, ad in reqs]
        _wait(iqa, srv, hs)
        for h, (rid, NT, seed, drop, add) in zip(hs, reqs):
            N = dict(REFS)[rid]
            T = N // NT
            assert iqa.iqa_poll(srv, h, 0) == iqa.IQA_OK
            l, a = _result(iqa, srv, h, T)
            x = synth.render_epoch(cats[rid], 500 + rid, dtype="f16")
            y = synth.render_epoch(cats[rid], seed, drop=drop, add=add, dtype="f16")
            ol, oa, osum = parity.oracle_maps(orc, x, y, NT, PARAMS)
            parity.assert_parity((l, a, None), (ol, oa, osum), PARAMS)
        # every step's two kernels were timed by the marks around them
        st = iqa.iqa_server_get_stats(srv)
        assert st.mean_step_generator_ms > 0 and st.mean_step_map_ms > 0
        assert st.generator_ms_per_pair <= st.mean_step_generator_ms
        assert st.map_ms_per_pair <= st.mean_step_map_ms
    finally:
        iqa.iqa_server_destroy(srv)


def test_same_result_alone_and_in_the_mix(ctx):
    """A request's maps are bit-identical when it is served alone and when it
    shares steps with a burst of other requests of different sizes."""
    from paper_2501_10653_gb300 import iqa
    srv, cats = _server(ctx, iqa.IQA_F16)
    try:
        probe = iqa.make_request(1, 64, 4242, [0, 2], (3, 10, 900, 0.3))
        h = iqa.iqa_submit(srv, probe)
        _wait(iqa, srv, [h])
        alone = _result(iqa, srv, h, 16)
        burst = []
        for i in range(30):
            rid = i % 3
            burst.append(iqa.iqa_submit(srv, iqa.make_request(rid, (32, 64, 128)[i % 3],
                                                              9000 + i, [i % 4])))
            if i == 13:
                h2 = iqa.iqa_submit(srv, probe)
        _wait(iqa, srv, burst + [h2])
        mixed = _result(iqa, srv, h2, 16)
        assert np.array_equal(alone[0], mixed[0]) and np.array_equal(alone[1], mixed[1])
        st = iqa.iqa_server_get_stats(srv)
        assert st.completed == 32 and st.mean_pairs_per_step > 1.0
    finally:
        iqa.iqa_server_destroy(srv)


def test_one_pair_per_launch_baseline_against_oracle(ctx, orc):
    from paper_2501_10653_gb300 import iqa
    srv, cats = _server(ctx, iqa.IQA_F32, one_pair_per_launch=1, time_kernels=1)
    try:
        reqs = [(0, 64, 31, [1]), (2, 32, 32, [0, 3]), (1, 128, 33, [])]
        hs = [iqa.iqa_submit(srv, iqa.make_request(r, nt, sd, dr)) for r, nt, sd, dr in reqs]
        _wait(iqa, srv, hs)
        for h, (rid, NT, seed, drop) in zip(hs, reqs):
            N = dict(REFS)[rid]
            l, a = _result(iqa, srv, h, N // NT)
            x = synth.render_epoch(cats[rid], 500 + rid)
            y = synth.render_epoch(cats[rid], seed, drop=drop)
            ol, oa, osum = parity.oracle_maps(orc, x, y, NT, PARAMS)
            parity.assert_parity((l, a, None), (ol, oa, osum), PARAMS)
        st = iqa.iqa_server_get_stats(srv)
        assert st.mean_pairs_per_step == pytest.approx(1.0)
        assert st.mean_step_generator_ms > 0 and st.mean_step_map_ms > 0
    finally:
        iqa.iqa_server_destroy(srv)


def test_small_pool_serialises_but_serves_everything(ctx):
    from paper_2501_10653_gb300 import iqa
    srv, _ = _server(ctx, iqa.IQA_F16, pool_bytes=9 << 20)  # one 2048^2 FP16 epoch
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(2, 64, 70 + i)) for i in range(5)]
        _wait(iqa, srv, hs)
        assert all(iqa.iqa_poll(srv, h, 0) == iqa.IQA_OK for h in hs)
        st = iqa.iqa_server_get_stats(srv)
        assert st.pool_peak_bytes <= 9 << 20
        with pytest.raises(iqa.IqaError) as ei:
            big = iqa.iqa_server_create(ctx, dtype=iqa.IQA_F16, pool_bytes=1 << 20,
                                        max_pairs_per_step=2, max_inflight_steps=1)
            try:
                iqa.iqa_server_add_reference(big, 0, synth.serving_catalog(1024, 0), 1)
                iqa.iqa_submit(big, iqa.make_request(0, 64, 1))
            finally:
                iqa.iqa_server_destroy(big)
        assert ei.value.status == iqa.IQA_ERR_NOMEM
    finally:
        iqa.iqa_server_destroy(srv)


def test_device_stall_is_reported_and_the_context_recovers(ctx, orc):
    """Fault injection without a GPU fault: the persistent kernel's producer
    issues nothing, so its consumers' bounded waits run out (20 ms); the step
    reports IQA_ERR_TIMEOUT through iqa_poll.  A server made after the
    injection is switched off serves correctly on the same context."""
    from paper_2501_10653_gb300 import iqa
    iqa.iqa_set_option(ctx, iqa.IQA_OPT_WAIT_TIMEOUT_US, 20_000)
    iqa.iqa_set_option(ctx, iqa.IQA_OPT_INJECT_STALL, 1)
    try:
        srv, _ = _server(ctx, iqa.IQA_F16)
    finally:
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_INJECT_STALL, 0)
        iqa.iqa_set_option(ctx, iqa.IQA_OPT_WAIT_TIMEOUT_US, 1_000_000)
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(0, 64, i)) for i in range(3)]
        _wait(iqa, srv, hs)
        assert all(iqa.iqa_poll(srv, h, 0) == iqa.IQA_ERR_TIMEOUT for h in hs)
        assert iqa.iqa_server_get_stats(srv).failed == 3
    finally:
        iqa.iqa_server_destroy(srv)
    srv, cats = _server(ctx, iqa.IQA_F16)
    try:
        h = iqa.iqa_submit(srv, iqa.make_request(0, 64, 5, [1]))
        _wait(iqa, srv, [h])
        l, a = _result(iqa, srv, h, 8)
        x = synth.render_epoch(cats[0], 500, dtype="f16")
        y = synth.render_epoch(cats[0], 5, drop=[1], dtype="f16")
        parity.assert_parity((l, a, None), parity.oracle_maps(orc, x, y, 64, PARAMS), PARAMS)
    finally:
        iqa.iqa_server_destroy(srv)


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_render_epoch_matches_host_mirror_bitwise(ctx, dt):
    """The public generator entry point, with drops and a transient."""
    import torch
    from paper_2501_10653_gb300 import iqa
    cat = synth.serving_catalog(1024, 3)
    out = torch.empty(1024 * 1024, dtype={"f32": torch.float32, "f16": torch.float16,
                                          "bf16": torch.bfloat16}[dt], device="cuda")
    iqa.iqa_render_epoch(ctx, cat, 987654321, out, DT[dt], drop=[1, 4], add=(2, 500, 17, 0.3))
    got = out.cpu().view(torch.int16 if dt != "f32" else torch.int32).numpy()
    want = synth.render_epoch(cat, 987654321, drop=[1, 4], add=(2, 500, 17, 0.3), dtype=dt)
    assert np.array_equal(got.view(np.uint8), want.reshape(-1).view(np.uint8))
