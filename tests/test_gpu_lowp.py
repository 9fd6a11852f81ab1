"""Reduced storage (PCE_FLAG_LOWP_STORAGE): bfloat16 windows, FP16 spectra with a
per-term power-of-two scale, FP32 arithmetic.

Two checks:
* Against the rounded operator: the oracle applied to the bfloat16-rounded
  windows and the plan's (rounded) spectra must match to the FP32 bar
  (1e-5): the conversions in the kernels are exact.
* Against the original FP64 operator: the storage rounding costs at most
  3e-3 relative l2, the bar for reduced storage; the measured error is
  printed per workload.
"""
import numpy as np
import pytest

import synth
from oracle import expansion as E


TOL_FP32 = 1e-5
TOL_LOWP = 3e-3


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_1604_04374_gb300 import build
    build.build()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(got, ref):
    got = np.asarray(got, np.float64).reshape(got.shape[0], -1)
    ref = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def test_bf16_helper():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie (to even: 1), 1 + 3 * 2^-9 rounds up
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 3.14159, 0.0], np.float32)
    r = bf16_round(x)
    assert list(r[:3]) == [1.0, 1.0, 1.0 + 2 ** -7]
    assert r[3] == 3.140625 and r[4] == 0.0


@pytest.mark.gpu
@pytest.mark.parametrize("shape,m,batch", [((64, 64), 4, 2), ((1024, 32), 4, 2), ((32, 128), 8, 1),
                                           ((1024,), 8, 2), ((256,), 4, 1)])
def test_lowp_matches_rounded_operator_and_bar(torch_cuda, shape, m, batch):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    from paper_1604_04374_gb300.pce import PCE_FLAG_LOWP_STORAGE
    if len(shape) == 2:
        pr = synth.problem_2d(shape[0], shape[1], m, batch, 600 + m, "normal")
    else:
        pr = synth.problem_1d(shape[0], m, batch, 600 + m)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=PCE_FLAG_LOWP_STORAGE)
    u = dev(torch, pr.u)
    y = plan.apply(u).cpu().numpy()
    x = plan.apply_adjoint(u).cpu().numpy()
    hhat = plan.hhat().cpu().numpy().astype(np.complex128)
    wr = bf16_round(pr.w)
    # the rounded operator, evaluated by the oracle
    yr = E.apply_from_spectra(pr.u, wr, hhat, shape)
    assert rel_l2(y, yr) < TOL_FP32
    # adjoint: transpose of the rounded operator, through the dense form on small sizes
    v = np.random.default_rng(1).standard_normal(pr.u.shape).astype(np.float32)
    xv = plan.apply_adjoint(dev(torch, v)).cpu().numpy().astype(np.float64)
    lhs = np.sum(yr * v)
    rhs = np.sum(pr.u.astype(np.float64) * xv)
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(yr ** 2) * np.sum(v.astype(np.float64) ** 2))
    # against the original operator: within the reduced-storage bar
    ey = rel_l2(y, E.apply(pr.u, pr.w, pr.h))
    ex = rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h))
    print(f"reduced storage {shape} m={m}: rel l2 forward {ey:.2e}, adjoint {ex:.2e}")
    assert ey < TOL_LOWP and ex < TOL_LOWP


@pytest.mark.gpu
def test_lowp_precision_workload_2048(torch_cuda):
    """2048 x 2048, B = 4, m = 64 hats on 8 x 8 nodes: reduced storage vs FP32 storage, sampled."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    from paper_1604_04374_gb300.pce import PCE_FLAG_LOWP_STORAGE
    pr = synth.workload("2d_2048_m64_b4")
    u = dev(torch, pr.u)
    rng = np.random.default_rng(4)
    pts = np.stack([rng.integers(0, n, 200) for n in pr.shape], axis=-1)
    sel = (slice(None),) + tuple(pts.T)
    yr = E.apply_at(pr.u, pr.w, pr.h, pts)
    xr = E.apply_adjoint_at(pr.u, pr.w, pr.h, pts)
    errs = {}
    for name, flags in (("fp32", 0), ("lowp", PCE_FLAG_LOWP_STORAGE)):
        plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=flags)
        y = plan.apply(u)[sel].cpu().numpy()
        x = plan.apply_adjoint(u)[sel].cpu().numpy()
        errs[name] = (rel_l2(y, yr), rel_l2(x, xr))
        plan.close()
    print("2048^2 m=64 B=4 rel l2 (forward, adjoint):", errs)
    assert max(errs["fp32"]) < TOL_FP32
    assert max(errs["lowp"]) < TOL_LOWP


@pytest.mark.gpu
def test_lowp_restrictions(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, PceError, pce
    pr = synth.problem_2d(32, 32, 4, 1, 5)
    with pytest.raises(PceError) as e:
        Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_LOWP_STORAGE | pce.PCE_FLAG_UNFUSED)
    assert e.value.status == pce.PCE_ERR_INVALID
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_LOWP_STORAGE)
    u = dev(torch, pr.u)
    with pytest.raises(PceError) as e:
        plan.backward(u, u.clone())
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
