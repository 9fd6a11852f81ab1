"""pce_apply_noalloc: the forward apply for callers that cannot allocate device memory.

The entry point runs the 2D forward kernels with their intermediates in the
library's static 64 MiB device block instead of the plan's scratch, and must
give the same result as pce_apply.  It is compared with pce_apply through the
C ABI on two calls in a row (the second call finds the first call's data in
the static block).  This file sorts last so that a stop at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_1604_04374_gb300 import build
    build.build()
    torch.cuda.init()
    return torch


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).double()
    b = b.reshape(b.shape[0], -1).double()
    return float(((a - b).norm(dim=1) / b.norm(dim=1)).max())


@pytest.mark.parametrize("name,args", [
    ("256x256_m16_b3", (256, 256, 16, 3, 31, "normal")),
    ("1024x1024_m16_b2", (1024, 1024, 16, 2, 32, "uniform")),
    ("64x512_m8_b5", (64, 512, 8, 5, 33, "normal")),
])
def test_noalloc_matches_apply_on_two_calls(torch_cuda, name, args):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce_apply, pce_apply_noalloc
    pr = synth.problem_2d(*args)
    dev = torch.device("cuda", 0)
    plan = Plan(torch.from_numpy(pr.w).to(dev), h=torch.from_numpy(pr.h).to(dev))
    stream = torch.cuda.current_stream().cuda_stream
    u1 = torch.from_numpy(pr.u).to(dev)
    u2 = torch.flip(u1, dims=[0, -1]).contiguous() * 2.0 - 0.5
    for u in (u1, u2):                       # two calls in a row on the shared static block
        ref = torch.empty_like(u)
        got = torch.full_like(u, float("nan"))
        pce_apply(plan.handle, u.data_ptr(), ref.data_ptr(), u.shape[0], stream)
        pce_apply_noalloc(plan.handle, u.data_ptr(), got.data_ptr(), u.shape[0], stream)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert _rel(got, ref) < TOL
    plan.close()


def test_noalloc_rejects_what_does_not_fit(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, PceError, pce, pce_apply_noalloc
    dev = torch.device("cuda", 0)
    # 2048 x 2048, m = 64: about 285 MB of scratch per right-hand side, more than 64 MiB
    pr = synth.problem_2d(2048, 2048, 64, 1, 34, "normal", (8, 8))
    plan = Plan(torch.from_numpy(pr.w).to(dev), h=torch.from_numpy(pr.h).to(dev))
    u = torch.from_numpy(pr.u).to(dev)
    y = torch.empty_like(u)
    with pytest.raises(PceError) as e:
        pce_apply_noalloc(plan.handle, u.data_ptr(), y.data_ptr(), 1, 0)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    assert "static scratch" in str(e.value)
    plan.close()
    # 1D plans have no scratch to place
    p1 = synth.problem_1d(256, 4, 1, 35)
    plan1 = Plan(torch.from_numpy(p1.w).to(dev), h=torch.from_numpy(p1.h).to(dev))
    u1 = torch.from_numpy(p1.u).to(dev)
    with pytest.raises(PceError) as e:
        pce_apply_noalloc(plan1.handle, u1.data_ptr(), torch.empty_like(u1).data_ptr(), 1, 0)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    plan1.close()
