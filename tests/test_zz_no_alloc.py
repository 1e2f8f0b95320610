"""The allocation-free divergence entry point against the context's own
divergence stage.

bfibm_divergence_noalloc serves callers that cannot let the library allocate
device memory (another allocator already owns it, a fixed budget must never
run out after start-up, or cudaMalloc's device-wide synchronisation is too
costly). It must give what BFIBM_STAGE_DIVERGENCE gives, call after call,
while reusing one fixed scratch array. This file sorts last so that a run
stopping at its first failure has already run every other test."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

from helpers import assert_close, cell_mask, face_mask

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the single-stage tolerance of the other GPU tests


@pytest.mark.parametrize("case", ["duct", "c1"])
def test_noalloc_divergence_matches_stage_twice(case):
    import torch
    if case == "duct":
        prm = W.base_params(3, (24, 20, 40), (0, 0, 1), 2, 1.0 / 24, sigma=0.7, euler=3.0)
    else:
        prm = W.c1()["params"]
    ctx = bfibm.Context(prm)
    rng = np.random.default_rng(21)
    for call in range(2):
        us = [np.where(face_mask(ctx, d), rng.normal(size=ctx.shape()), 0.0)
              for d in range(ctx.dim)]
        for d in range(ctx.dim):
            ctx.set_field("ut", us[d], d)
        ctx.stage("divergence")
        ref = ctx.get_field("prhs")
        dev = [torch.from_numpy(u).cuda() for u in us]
        b = torch.zeros(ctx.shape(), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        bfibm.divergence_noalloc(prm, [t.data_ptr() for t in dev], b.data_ptr(), stream)
        torch.cuda.synchronize()
        got = b.cpu().numpy()
        cm = cell_mask(ctx)
        assert_close(got[cm], ref[cm], TOL, "no-alloc divergence, call %d" % call)
        assert abs(got[cm].mean()) < 1e-12 * np.abs(got[cm]).max()
    ctx.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    prm = W.base_params(3, (512, 256, 256), (0, 0, 1), 2, 1.0 / 512)   # 2^25 cells
    with pytest.raises(bfibm.BfibmError) as e:
        bfibm.divergence_noalloc(prm, [1, 1, 1], 1)
    assert e.value.status == bfibm.EINVAL
