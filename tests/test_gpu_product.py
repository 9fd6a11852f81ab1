"""GPU parity of the product-convolution form P_m u = sum_k w_k . (h_k * u)
(PCE_FLAG_PRODUCT_CONVOLUTION) against the FP64 oracle (O6 and its adjoint).

Bar: relative l2 <= 1e-5 with FP32 storage, <= 3e-3 with reduced storage.
"""
import numpy as np
import pytest

import synth
from oracle import dft as D
from oracle import expansion as E

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_1604_04374_gb300 import build
    build.build()
    torch.cuda.init()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(got, ref):
    got = got.reshape(got.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def problem(shape, m, batch, seed):
    if len(shape) == 1:
        return synth.problem_1d(shape[0], m, batch, seed)
    return synth.problem_2d(shape[0], shape[1], m, batch, seed, "normal")


def short_problem(n, m, batch, seed, radius=24):
    rng = np.random.default_rng(seed)
    w = synth.hat_windows_1d(n, m).astype(np.float32)
    h = np.zeros((m, n), np.float32)
    offs = np.arange(-radius, radius + 1) % n
    h[:, offs] = rng.standard_normal((m, offs.size)).astype(np.float32)
    u = rng.standard_normal((batch, n)).astype(np.float32)
    return synth.Problem("short", (n,), m, w, h, u)


CASES = [((64,), 4, 2), ((1024,), 8, 1), ((4096,), 4, 2), ((32, 64), 4, 2), ((64, 64), 16, 1),
         ((16, 1024), 4, 2), ((1024, 16), 4, 1), ((128, 256), 8, 1)]


@pytest.mark.parametrize("shape,m,batch", CASES)
def test_product_convolution_matches_oracle(torch_cuda, shape, m, batch):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = problem(shape, m, batch, 700 + m + batch)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_PRODUCT_CONVOLUTION)
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.product_convolution(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.product_convolution_adjoint(pr.u, pr.w, pr.h)) < TOL
    # the exported spectra are those of h_k, as for any plan
    got = plan.hhat().cpu().numpy().astype(np.complex128)
    ref = np.stack([D.rdft_nd(pr.h[k].astype(np.float64), len(shape)) for k in range(m)])
    if len(shape) == 1:
        ref[:, 0] = ref[:, 0].real
        ref[:, -1] = ref[:, -1].real
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-6


@pytest.mark.parametrize("n,m", [(1 << 14, 3), (1 << 16, 4)])
def test_product_convolution_large_1d(torch_cuda, n, m):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = short_problem(n, m, 2, 90 + m)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_PRODUCT_CONVOLUTION)
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.product_convolution(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.product_convolution_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_product_convolution_from_spectra_unfused_and_lowp(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = problem((64, 128), 4, 2, 71)
    F = pce.PCE_FLAG_PRODUCT_CONVOLUTION
    ref_y = E.product_convolution(pr.u, pr.w, pr.h)
    ref_x = E.product_convolution_adjoint(pr.u, pr.w, pr.h)
    u = dev(torch, pr.u)
    hhat = np.stack([np.fft.rfft2(pr.h[k].astype(np.float64)) for k in range(4)]).astype(np.complex64)
    p1 = Plan(dev(torch, pr.w), hhat=dev(torch, hhat), flags=F)
    assert rel(host(p1.apply(u)), ref_y) < TOL
    assert rel(host(p1.apply_adjoint(u)), ref_x) < TOL
    p2 = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=F | pce.PCE_FLAG_UNFUSED)
    assert rel(host(p2.apply(u)), ref_y) < TOL
    assert rel(host(p2.apply_adjoint(u)), ref_x) < TOL
    p3 = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=F | pce.PCE_FLAG_LOWP_STORAGE)
    assert rel(host(p3.apply(u)), ref_y) < 3e-3
    assert rel(host(p3.apply_adjoint(u)), ref_x) < 3e-3


def test_product_convolution_in_batches_and_restrictions(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, apply_batch, pce
    from paper_1604_04374_gb300.pce import PceError
    pr = problem((32, 64), 4, 1, 72)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_PRODUCT_CONVOLUTION)
    u = dev(torch, pr.u)
    y = torch.empty_like(u)
    x = torch.empty_like(u)
    apply_batch([(plan, u, y, False), (plan, u, x, True)])
    torch.cuda.synchronize()
    assert rel(host(y), E.product_convolution(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(x), E.product_convolution_adjoint(pr.u, pr.w, pr.h)) < TOL
    assert plan.launch_count(False, 1) == 3 and plan.launch_count(True, 1) == 3
    with pytest.raises(PceError) as e:
        plan.backward(u, u)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    with pytest.raises(PceError) as e:
        pce.pce_apply_noalloc(plan.handle, u.data_ptr(), y.data_ptr(), 1, 0)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
