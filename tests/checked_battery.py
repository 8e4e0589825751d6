"""A battery of launches for the bounds-checked library (libiqa_checked.so):
every kernel family over the launch shapes the tests use, with the failed-check
count read after each group.  Run in its own process with IQA_LIBRARY set (see
test_gpu_checked_build.py); prints one line per group and exits non-zero on the
first group with a failed check or a wrong map."""
import sys

import numpy as np

import parity
from paper_2501_10653_gb300 import iqa, synth

PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}


def _violations(what):
    n = iqa.iqa_debug_violations()
    print("%-40s failed checks: %d" % (what, n), flush=True)
    if n:
        sys.exit(1)


def main():
    import torch
    import oracle
    orc = oracle.Oracle()
    ctx = iqa.iqa_create(0, 0)
    st = torch.cuda.current_stream()
    _violations("start")

    # one-pair kernel: default and explicit shapes, every storage type
    shapes = [(512, 16), (512, 64), (1024, 256), (480, 48), (384, 128), (96, 96), (250, 10)]
    for dt in ("f32", "f16", "bf16"):
        for N, NT in shapes:
            x, y = synth.paper_pair(N=N, dtype=dt)
            got = parity.gpu_maps(ctx, x, y, NT, PARAMS)
            if dt == "f32" and N == 512:
                parity.assert_parity(got, parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)
    x, y = synth.paper_pair(N=512)
    for cfg in (dict(variant=0, threads=128, ilp=8, split=2), dict(variant=0, threads=256,
                ilp=4, split=4), dict(variant=0, threads=512, ilp=2, split=8),
                dict(variant=0, threads=128, ilp=4, tiles_across=2)):
        iqa.iqa_set_config(ctx, iqa.IQA_F32, 512, 64, iqa.MAPS_BOTH, cfg)
        parity.gpu_maps(ctx, x, y, 64, PARAMS)
    iqa.iqa_set_config(ctx, iqa.IQA_F32, 512, 64, iqa.MAPS_BOTH, None)
    # misaligned pointers take the scalar path
    base = torch.from_numpy(np.concatenate([[0.0], x.ravel(), y.ravel()]).astype(np.float32)).cuda()
    iqa.iqa_both(ctx, base[1:].data_ptr(), base[1 + 512 * 512:].data_ptr(), iqa.IQA_F32, 512,
                 64, PARAMS, torch.empty(64, device="cuda"), torch.empty(64, device="cuda"),
                 None, st)
    torch.cuda.synchronize()
    _violations("one-pair kernel")

    # persistent kernel: explicit shapes through the one-pair entry point
    for dt in ("f32", "f16"):
        x, y = synth.paper_pair(N=512, dtype=dt)
        code = parity.dtype_code(x)
        for NT in (16, 64, 256):
            for cfg in (dict(variant=1, threads=128, stages=2, stage_kb=16, ctas_per_sm=3),
                        dict(variant=1, threads=256, stages=4, stage_kb=4, ctas_per_sm=1),
                        dict(variant=1, threads=512, stages=3, stage_kb=2, ctas_per_sm=2)):
                try:
                    iqa.iqa_set_config(ctx, code, 512, NT, iqa.MAPS_BOTH, cfg)
                except iqa.IqaError:
                    continue
                parity.gpu_maps(ctx, x, y, NT, PARAMS)
            iqa.iqa_set_config(ctx, code, 512, NT, iqa.MAPS_BOTH, None)
    _violations("persistent kernel, one pair")

    # batched plans: mixed sizes (wide 3-D units where N allows), FP32 and FP16
    specs = [(1024, 16), (256, 32), (512, 128), (1024, 32), (512, 64), (768, 96), (2048, 64)]
    for dt, code in (("f32", iqa.IQA_F32), ("f16", iqa.IQA_F16)):
        keep, pairs = [], []
        for i, (N, NT) in enumerate(specs):
            x, y = synth.mixed_batch_pair(i, N, dtype=dt)
            dx, dy = parity.to_device(x), parity.to_device(y)
            T = N // NT
            o = (torch.empty(T * T, device="cuda"), torch.empty(T * T, device="cuda"))
            keep.append((dx, dy, o, x, y, NT))
            pairs.append(iqa.make_pair(dx, dy, N, NT, *o))
        plan = iqa.iqa_plan_create(ctx, pairs, code, PARAMS, iqa.IQA_PLAN_GRAPH)
        iqa.iqa_plan_autotune(plan, st, 1)
        for _ in range(2):
            iqa.iqa_plan_launch(plan, st)
        torch.cuda.synchronize()
        iqa.iqa_plan_destroy(plan)
        dx, dy, o, x, y, NT = keep[0]
        parity.assert_parity((o[0].cpu().numpy(), o[1].cpu().numpy(), None),
                             parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)
        iqa.iqa_batch_noalloc(pairs[:5], code, PARAMS, st)
        torch.cuda.synchronize()
    _violations("batched plans and no-alloc batches")

    # batched plans whose units span several tile rows (explicit shapes)
    for N, NT, dt, th, kpx in ((1024, 16, "f32", 128, 32), (288, 16, "f32", 128, 32),
                               (2048, 32, "f32", 256, 64), (768, 16, "f16", 128, 32),
                               (512, 8, "f32", 128, 64), (2048, 64, "f32", 128, 64)):
        x, y = synth.mixed_batch_pair(1, N, dtype=dt)
        dx, dy = parity.to_device(x), parity.to_device(y)
        T = N // NT
        o = (torch.empty(T * T, device="cuda"), torch.empty(T * T, device="cuda"),
             torch.empty((T * T, 4), dtype=torch.float64, device="cuda"))
        plan = iqa.iqa_plan_create(ctx, [iqa.make_pair(dx, dy, N, NT, *o)],
                                   parity.dtype_code(x), PARAMS, iqa.IQA_PLAN_INDEPENDENT)
        iqa.iqa_plan_set_config(plan, {"threads": th, "unit_kpx": kpx})
        for _ in range(2):
            iqa.iqa_plan_launch(plan, st)
        torch.cuda.synchronize()
        iqa.iqa_plan_destroy(plan)
        parity.assert_parity(tuple(t.cpu().numpy() for t in o),
                             parity.oracle_maps(orc, x, y, NT, PARAMS), PARAMS)
    _violations("plans of several tile rows per unit")

    # Eq. 3 / Eq. 4 merge: thread, warp and cluster shapes
    x, y = synth.paper_pair(N=1024)
    _, _, sums = parity.gpu_maps(ctx, x, y, 8, PARAMS)
    ds = torch.from_numpy(sums).cuda()
    for m in (2, 4, 16, 64, 128):
        M = 128 // m
        iqa.iqa_merge(ctx, ds, 128, m, PARAMS, torch.empty(M * M, device="cuda"),
                      torch.empty(M * M, device="cuda"), None, st)
    torch.cuda.synchronize()
    _violations("merge kernels")

    # device generator and the serving loop (unbanded steps, several grids)
    cat = synth.serving_catalog(512, 3)
    for code, tdt in ((iqa.IQA_F32, torch.float32), (iqa.IQA_F16, torch.float16)):
        out = torch.empty(512 * 512, dtype=tdt, device="cuda")
        iqa.iqa_render_epoch(ctx, cat, 11, out, code, drop=[1], add=(0, 500, 3, 0.5))
    srv = iqa.iqa_server_create(ctx, dtype=iqa.IQA_F16, max_pairs_per_step=8,
                                max_inflight_steps=2, pool_bytes=1 << 30, params=PARAMS)
    try:
        for rid, N in ((0, 512), (1, 2048), (2, 4096)):
            iqa.iqa_server_add_reference(srv, rid, synth.serving_catalog(N, rid), 5 + rid)
        hs = [iqa.iqa_submit(srv, iqa.make_request(i % 3, (32, 64, 128)[i % 3], 100 + i,
                                                   [i % 2])) for i in range(12)]
        for h in hs:
            while iqa.iqa_poll(srv, h, 200_000) == iqa.IQA_PENDING:
                pass
            assert iqa.iqa_poll(srv, h, 0) == iqa.IQA_OK
    finally:
        iqa.iqa_server_destroy(srv)
    _violations("generator and serving loop")
    iqa.iqa_destroy(ctx)
    print("checked battery: no failed checks", flush=True)


if __name__ == "__main__":
    main()
