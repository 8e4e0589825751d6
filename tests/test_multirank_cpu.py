"""The N>1 path of bench.py on the CPU: two ranks over gloo (no GPU).

The map computation shards with no data-path collective (every pair and tile
is independent), so `bench.py --gpus N` runs N replicas on distinct pairs and
only reduces its timing and byte counts across ranks.  These tests run those
reductions and the rank-distinct input selection in two real processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    r, w, local = bench.dist_env()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    t = bench.max_over_ranks(1.5 + rank, w)          # per-rank timings
    b = bench.sum_over_ranks(100.0 * (rank + 1), w)  # per-rank bytes
    x, _ = bench._pool_pairs(r, 1)[0]
    out[rank] = (r, w, t, b, float(x[0, 0]), float(x.sum()))
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_timing_reductions_and_distinct_inputs():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    r0, r1 = out[0], out[1]
    assert (r0[0], r0[1]) == (0, 2) and (r1[0], r1[1]) == (1, 2)
    # the timing is the max over ranks, the work the sum, on every rank
    assert r0[2] == r1[2] == 2.5
    assert r0[3] == r1[3] == 300.0
    # each rank streams its own pairs (independent replicas)
    assert r0[5] != r1[5]


def _reference_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    res = bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "2",
                                                "--warmup", "3"]))
    out[rank] = res


@pytest.mark.timeout(300)
def test_reference_arm_prints_on_rank_zero_only():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_reference_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    assert out[1] is None
    res = out[0]
    assert res["impl"] == "reference" and res["value"] > 0 and res["n_gpus"] == 2
    assert res["e2e"]["h2d_bytes_per_step"] == 0 and res["cpu_baseline"]["kind"] == "oracle"
