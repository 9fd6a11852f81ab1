"""pce_apply_noalloc: the forward apply for callers that cannot allocate device memory.

The entry point runs the 2D forward kernels with their intermediates in the
library's static 64 MiB device block instead of the plan's scratch, and must
give the same result as pce_apply.  It is compared through the C ABI with
pce_apply on two calls in a row (the second call finds the first call's data
in the static block) and with the FP64 oracle, for dense FP32 plans, plans
with reduced storage, separable and sectioned plans (which it runs on their
whole-grid structures) and a plan with 2048-point columns.  This file sorts
last so that a stop at the first failure has already run every other test.
"""
import numpy as np
import pytest

import synth
from oracle import direct as C

pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_LOWP = 3e-3


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


def _rel_np(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


CASES = [
    ("256x256_m16_b3", (256, 256, 16, 3, 31, "normal"), "dense"),
    ("1024x1024_m16_b2", (1024, 1024, 16, 2, 32, "uniform"), "dense"),
    ("64x512_m8_b5", (64, 512, 8, 5, 33, "normal"), "dense"),
    ("256x256_m16_b3_lowp", (256, 256, 16, 3, 36, "normal"), "lowp"),
    ("1024x128_m16_b2_separable", (1024, 128, 16, 2, 37, "uniform"), "separable"),
    ("1024x256_m16_b2_sectioned", (1024, 256, 16, 2, 38, "normal"), "sectioned"),
    ("2048x256_m4_b2", (2048, 256, 4, 2, 39, "normal"), "dense"),
]


@pytest.mark.parametrize("name,args,kind", CASES)
def test_noalloc_matches_apply_on_two_calls(torch_cuda, name, args, kind):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce, pce_apply, pce_apply_noalloc
    pr = synth.problem_2d(*args)
    dev = torch.device("cuda", 0)
    h = torch.from_numpy(pr.h).to(dev)
    if kind == "separable":
        wy, wx = synth.hat_factors_2d(pr.shape[0], pr.shape[1], *pr.meta["grid"])
        plan = Plan(wy=torch.from_numpy(wy).to(dev), wx=torch.from_numpy(wx).to(dev), h=h)
        assert plan.slots() > 0
    else:
        flags = {"dense": 0, "lowp": pce.PCE_FLAG_LOWP_STORAGE, "sectioned": pce.PCE_FLAG_SECTIONED}[kind]
        plan = Plan(torch.from_numpy(pr.w).to(dev), h=h, flags=flags)
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
        # same storage precision on both sides: equal up to rounding order
        assert _rel(got, ref) < TOL
        # and the operator itself, against the FP64 oracle (every output)
        yo = C.apply(u.cpu().numpy(), pr.w, pr.h)
        assert _rel_np(got.double().cpu().numpy(), yo) < (TOL_LOWP if kind == "lowp" else TOL)
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
