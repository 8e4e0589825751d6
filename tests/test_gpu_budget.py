"""The context's device-memory budget (iqa_create's hbm_budget_bytes): every
allocation the library makes on the context's behalf is refused with
IQA_ERR_NOMEM when it would exceed the budget, before anything is allocated,
and the context stays usable (needs a GPU)."""
import numpy as np
import pytest

import parity
from paper_2501_10653_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}


def test_budget_refuses_workspace_tables_and_pool(orc):
    import torch
    from paper_2501_10653_gb300 import build, iqa
    build.build()
    ctx = iqa.iqa_create(0, 1 << 20)  # 1 MiB
    try:
        N, NT = 512, 64
        T = N // NT
        x, y = synth.paper_pair(N=N)
        hl = np.full(T * T, np.nan, np.float32)
        ha = np.full(T * T, np.nan, np.float32)
        # the host path stages both 1 MiB images on the device: over budget
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_both_host(ctx, x, y, iqa.IQA_F32, N, NT, PARAMS, hl, ha)
        assert ei.value.status == iqa.IQA_ERR_NOMEM
        assert "budget" in iqa.iqa_last_error(ctx)
        assert np.all(np.isnan(hl))
        # plan tables of 3000 descriptors (384 B each): over budget
        dx, dy = parity.to_device(x), parity.to_device(y)
        lm = torch.empty(T * T, device="cuda")
        am = torch.empty(T * T, device="cuda")
        pair = iqa.make_pair(dx, dy, N, NT, lm, am)
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_plan_create(ctx, [pair] * 3000, iqa.IQA_F32, PARAMS)
        assert ei.value.status == iqa.IQA_ERR_NOMEM
        # a serving pool above the budget
        with pytest.raises(iqa.IqaError) as ei:
            iqa.iqa_server_create(ctx, dtype=iqa.IQA_F16, pool_bytes=64 << 20,
                                  max_pairs_per_step=2, max_inflight_steps=1)
        assert ei.value.status == iqa.IQA_ERR_NOMEM
        # the context still serves what fits: device pointers (no workspace)
        # and a small plan
        iqa.iqa_both(ctx, dx, dy, iqa.IQA_F32, N, NT, PARAMS, lm, am, None,
                     torch.cuda.current_stream())
        torch.cuda.synchronize()
        want = parity.oracle_maps(orc, x, y, NT, PARAMS)
        parity.assert_parity((lm.cpu().numpy(), am.cpu().numpy(), None), want, PARAMS)
        plan = iqa.iqa_plan_create(ctx, [pair] * 4, iqa.IQA_F32, PARAMS)
        iqa.iqa_plan_destroy(plan)
    finally:
        iqa.iqa_destroy(ctx)
