"""Serving loop on the host only (no GPU): the native scheduler with a simulated
executor -- a step completes after its input bytes / a modelled bandwidth, or
never (a stalled completion source).  Covers admission by the pool budget,
arrival order, continuous batching, the host watchdog and bad arguments."""
import time

import pytest

from paper_2501_10653_gb300 import iqa, synth


@pytest.fixture(scope="module")
def lib():
    from paper_2501_10653_gb300 import build
    build.build()
    return iqa


def _server(lib, **kw):
    args = dict(dtype=iqa.IQA_F16, max_pairs_per_step=4, max_inflight_steps=2,
                pool_bytes=64 << 20, simulate=1, sim_bytes_per_s=20e9)
    args.update(kw)
    srv = iqa.iqa_server_create(None, **args)
    for rid, N in ((0, 512), (1, 1024), (2, 2048)):
        iqa.iqa_server_add_reference(srv, rid, synth.serving_catalog(N, rid), 100 + rid)
    return srv


def _wait_all(srv, hs, timeout_s=20.0):
    t0 = time.time()
    out = {}
    for h in hs:
        while True:
            st = iqa.iqa_poll(srv, h, 100_000)
            if st != iqa.IQA_PENDING:
                out[h] = st
                break
            assert time.time() - t0 < timeout_s, "request never finished"
    return out


def test_all_requests_complete_with_latency_stats(lib):
    srv = _server(lib)
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(i % 3, 64, 1000 + i)) for i in range(40)]
        sts = _wait_all(srv, hs)
        assert all(s == iqa.IQA_OK for s in sts.values())
        for h in hs:
            lat = iqa.iqa_result(srv, h)
            assert lat >= 0.0
        st = iqa.iqa_server_get_stats(srv)
        assert st.completed == 40 and st.failed == 0 and st.pending == 0
        assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms
        assert st.pairs_per_s > 0 and st.steps >= 10
    finally:
        iqa.iqa_server_destroy(srv)


def test_continuous_batching_fills_steps(lib):
    """A burst arriving while steps are in flight is admitted in later steps of
    several pairs each (not one queue entry per step)."""
    srv = _server(lib, sim_bytes_per_s=2e9, max_pairs_per_step=8)
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(0, 64, i)) for i in range(64)]
        _wait_all(srv, hs)
        st = iqa.iqa_server_get_stats(srv)
        assert st.completed == 64
        assert st.mean_pairs_per_step > 2.0
    finally:
        iqa.iqa_server_destroy(srv)


def test_admission_respects_pool_budget(lib):
    """A pool that holds one 2048^2 FP16 epoch (8 MB) admits one such request at
    a time; all still complete, and the peak pool use never exceeds the pool."""
    srv = _server(lib, pool_bytes=9 << 20, sim_bytes_per_s=5e9)
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(2, 64, i)) for i in range(6)]
        sts = _wait_all(srv, hs)
        assert all(s == iqa.IQA_OK for s in sts.values())
        st = iqa.iqa_server_get_stats(srv)
        assert st.pool_peak_bytes <= 9 << 20
        assert st.mean_pairs_per_step == pytest.approx(1.0)
    finally:
        iqa.iqa_server_destroy(srv)


def test_request_larger_than_pool_is_rejected(lib):
    srv = _server(lib, pool_bytes=4 << 20)
    try:
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_submit(srv, iqa.make_request(2, 64, 1))  # 8 MB epoch
        assert ei.value.status == iqa.IQA_ERR_NOMEM
        h = iqa.iqa_submit(srv, iqa.make_request(0, 64, 1))  # 0.5 MB fits
        assert _wait_all(srv, [h])[h] == iqa.IQA_OK
    finally:
        iqa.iqa_server_destroy(srv)


def test_arrival_order_is_kept(lib):
    """With one step slot and one pair per step, requests finish in arrival order."""
    srv = _server(lib, max_inflight_steps=1, max_pairs_per_step=1, sim_bytes_per_s=1e9)
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(i % 2, 64, i)) for i in range(8)]
        _wait_all(srv, hs)
        lats = [iqa.iqa_result(srv, h) for h in hs]
        # later arrivals wait behind earlier ones: latencies grow in order
        assert all(b >= a - 0.5 for a, b in zip(lats, lats[1:]))
    finally:
        iqa.iqa_server_destroy(srv)


def test_stalled_completion_source_hits_the_watchdog(lib):
    """Steps that never complete: polls come back IQA_PENDING until the host
    watchdog fails the step's requests with IQA_ERR_TIMEOUT; requests that
    could not start (every slot stuck) stay pending."""
    srv = _server(lib, simulate=2, max_inflight_steps=1, max_pairs_per_step=2,
                  step_timeout_ms=150.0)
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(0, 64, i)) for i in range(4)]
        assert iqa.iqa_poll(srv, hs[0], 0) == iqa.IQA_PENDING
        assert iqa.iqa_poll(srv, hs[0], 2_000_000) == iqa.IQA_ERR_TIMEOUT
        # the stuck step took hs[0] and, if it had arrived in time, hs[1]
        second = iqa.iqa_poll(srv, hs[1], 100_000)
        assert second in (iqa.IQA_ERR_TIMEOUT, iqa.IQA_PENDING)
        assert iqa.iqa_poll(srv, hs[2], 100_000) == iqa.IQA_PENDING
        assert iqa.iqa_poll(srv, hs[3], 0) == iqa.IQA_PENDING
        st = iqa.iqa_server_get_stats(srv)
        assert st.failed == (2 if second == iqa.IQA_ERR_TIMEOUT else 1)
        assert st.completed == 0
    finally:
        iqa.iqa_server_destroy(srv)


def test_bad_requests_and_config(lib):
    srv = _server(lib)
    try:
        for req in (iqa.make_request(9, 64, 1), iqa.make_request(0, 48, 1),
                    iqa.make_request(0, 1024, 1), iqa.make_request(0, 64, 1, drop=range(9)),
                    iqa.make_request(0, 64, 1, add=(999, 5, 5, 1.0))):
            with pytest.raises(iqa.IqaError) as ei:
                iqa.iqa_submit(srv, req)
            assert ei.value.status == iqa.IQA_ERR_INVALID_ARG
        assert iqa.iqa_poll(srv, 123456789, 0) == iqa.IQA_ERR_INVALID_ARG
        with pytest.raises(iqa.IqaError):
            iqa.iqa_server_add_reference(srv, 0, synth.serving_catalog(512, 0), 1)
    finally:
        iqa.iqa_server_destroy(srv)
    with pytest.raises(iqa.IqaError):
        iqa.iqa_server_create(None, max_pairs_per_step=65, simulate=1)
    with pytest.raises(iqa.IqaError):
        iqa.iqa_server_create(None, simulate=0)
    for bad in (dict(max_inflight_steps=9), dict(generator_blocks_per_sm=9),
                dict(generator_blocks_per_sm=-1), dict(map_ctas_per_sm=5),
                dict(time_kernels=2)):
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_server_create(None, simulate=1, **bad)
        assert ei.value.status == iqa.IQA_ERR_INVALID_ARG, bad
    # the new settings at their limits are accepted
    ok = iqa.iqa_server_create(None, simulate=1, max_inflight_steps=8,
                               generator_blocks_per_sm=8, map_ctas_per_sm=1, time_kernels=1)
    iqa.iqa_server_destroy(ok)


def test_step_byte_cap_splits_large_from_small(lib):
    """With a cap of 4 MB of input per step, a 2048^2 FP16 pair (16 MB) runs
    alone and the 512^2 pairs (1 MB each) are grouped up to four per step."""
    srv = _server(lib, max_pairs_per_step=16, max_step_bytes=4 << 20, sim_bytes_per_s=2e9)
    try:
        hs = [iqa.iqa_submit(srv, iqa.make_request(2, 64, 0))]
        hs += [iqa.iqa_submit(srv, iqa.make_request(0, 64, i)) for i in range(16)]
        _wait_all(srv, hs)
        st = iqa.iqa_server_get_stats(srv)
        assert st.completed == 17
        assert st.steps >= 5  # 1 large + at least 4 groups of <= 4 small
    finally:
        iqa.iqa_server_destroy(srv)


def test_native_trace_driver(lib):
    """iqa_server_run_trace submits at the given times and returns when all have
    finished; the statistics count every request and the wall time covers the
    trace."""
    srv = _server(lib, sim_bytes_per_s=50e9)
    try:
        reqs = [iqa.make_request(i % 3, 64, i) for i in range(100)]
        times = [0.002 * i for i in range(100)]
        t0 = time.time()
        iqa.iqa_server_run_trace(srv, reqs, times, 30.0)
        assert time.time() - t0 >= 0.198
        st = iqa.iqa_server_get_stats(srv)
        assert st.completed == 100 and st.pending == 0 and st.p99_ms > 0
    finally:
        iqa.iqa_server_destroy(srv)


def test_latency_split_adds_up(lib):
    """The statistics split each request's latency into queueing, the launch
    calls and the rest (device work, or here its modelled time); one request
    at a time, the parts' medians add up to the median latency and the rest
    matches the modelled step time.  Medians over 30 requests: the first few
    after set-up can wait for a core while the catalogue set-up's numpy
    threads wind down."""
    rate = 2e9  # 2 N^2 * 2 bytes of an N=1024 FP16 pair = 4 MiB -> about 2.1 ms
    srv = _server(lib, sim_bytes_per_s=rate)
    try:
        for i in range(30):
            h = iqa.iqa_submit(srv, iqa.make_request(1, 64, 300 + i))
            assert _wait_all(srv, [h])[h] == iqa.IQA_OK
        st = iqa.iqa_server_get_stats(srv)
        model_ms = 1e3 * 2 * 1024 * 1024 * 2 / rate
        assert st.completed == 30
        assert 0.0 <= st.p50_queue_ms < st.p50_ms and 0.0 <= st.p50_launch_ms < st.p50_ms
        # the modelled time runs from the start of the launch calls, the
        # device part from their end (microseconds later)
        assert model_ms - 0.05 <= st.p50_device_ms < model_ms + 2.0
        parts = st.p50_queue_ms + st.p50_launch_ms + st.p50_device_ms
        assert abs(parts - st.p50_ms) < 0.5
    finally:
        iqa.iqa_server_destroy(srv)
