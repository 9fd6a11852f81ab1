"""GPU gradients (pce_backward and the autograd Function) against the FP64 oracle.

The oracle's gradients (oracle.expansion.grad) are pinned by central finite
differences.  At the differentiation workload size (512 x 512, B = 16,
m = 16) the check is a property that holds at any size: the loss
L = <H_m u, r> is linear in w for fixed hhat and in hhat for fixed w, so
L(w + d) - L(w - d) = 2 <dL/dw, d> exactly (up to rounding), and likewise
for hhat and u.
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
    return t.detach().cpu().numpy()


def rel(got, ref):
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) else np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def _case(shape, m, batch, seed):
    if len(shape) == 2:
        pr = synth.problem_2d(shape[0], shape[1], m, batch, seed, "normal")
    else:
        pr = synth.problem_1d(shape[0], m, batch, seed)
    r = np.random.default_rng(seed + 1).standard_normal(pr.u.shape).astype(np.float32)
    return pr, r


@pytest.mark.parametrize("shape,m,batch", [((64, 64), 4, 2), ((32, 128), 8, 3), ((16, 16), 4, 1),
                                           ((16, 1024), 4, 2), ((1024, 16), 4, 1), ((512, 16), 4, 2),
                                           ((256,), 4, 3), ((1024,), 8, 2), ((64,), 3, 1)])
def test_backward_matches_oracle(torch_cuda, shape, m, batch):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    pr, r = _case(shape, m, batch, 500 + m + batch)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    du, dw, dh = plan.backward(dev(torch, pr.u), dev(torch, r))
    torch.cuda.synchronize()
    h64 = pr.h.astype(np.float64)
    rdu, rdw, _, rdh = E.grad(pr.u, pr.w, h64, r)
    assert rel(host(du), rdu) < TOL
    assert rel(host(dw), rdw) < TOL
    assert rel(host(dh), rdh) < TOL


def test_backward_with_non_hermitian_spectra(torch_cuda):
    """dL/dhhat does not depend on hhat; with a random complex hhat it still equals the oracle's."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    rng = np.random.default_rng(3)
    shape, m = (16, 32), 3
    w = rng.standard_normal((m,) + shape).astype(np.float32)
    hs = (m, 16, 17)
    hhat = (rng.standard_normal(hs) + 1j * rng.standard_normal(hs)).astype(np.complex64)
    u = rng.standard_normal((2,) + shape).astype(np.float32)
    r = rng.standard_normal((2,) + shape).astype(np.float32)
    plan = Plan(dev(torch, w), hhat=dev(torch, hhat))
    _, _, dh = plan.backward(dev(torch, u), dev(torch, r), need_u=False, need_w=False)
    h0 = np.zeros((m,) + shape)
    _, _, _, rdh = E.grad(u, w, h0, r)
    assert rel(host(dh), rdh) < TOL


def test_autograd_function(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import convolution_product
    pr, r = _case((32, 64), 4, 2, 77)
    hhat = np.stack([np.fft.rfft2(pr.h[k].astype(np.float64)) for k in range(4)]).astype(np.complex64)
    u = dev(torch, pr.u).requires_grad_(True)
    w = dev(torch, pr.w).requires_grad_(True)
    hh = dev(torch, hhat).requires_grad_(True)
    y = convolution_product(u, w, hh)
    loss = (y * dev(torch, r)).sum()
    loss.backward()
    rdu, rdw, _, rdh = E.grad(pr.u, pr.w, pr.h.astype(np.float64), r)
    assert rel(host(u.grad), rdu) < TOL
    assert rel(host(w.grad), rdw) < TOL
    assert rel(host(hh.grad), rdh) < TOL
    yr = E.apply(pr.u, pr.w, pr.h)
    assert rel(host(y), yr) < TOL


def test_differentiation_workload_linearity(torch_cuda):
    """512 x 512, B = 16, m = 16: exact directional derivatives of the bilinear loss."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    pr = synth.workload("2d_512_m16_b16")
    rng = np.random.default_rng(9)
    r = dev(torch, rng.standard_normal(pr.u.shape).astype(np.float32))
    w = dev(torch, pr.w)
    u = dev(torch, pr.u)
    base = Plan(w, h=dev(torch, pr.h))
    hhat = base.hhat()
    du, dw, dh = base.backward(u, r)

    def loss(ww, hh, uu):
        p = Plan(ww.contiguous(), hhat=hh.contiguous())
        val = torch.sum(p.apply(uu).double() * r.double()).item()
        p.close()
        return val

    dW = dev(torch, rng.standard_normal(pr.w.shape).astype(np.float32)) * 1.0
    fd = loss(w + dW, hhat, u) - loss(w - dW, hhat, u)
    an = 2 * torch.sum(dw.double() * dW.double()).item()
    assert abs(fd - an) <= 1e-4 * abs(an)
    dH = (torch.randn(hhat.shape, dtype=torch.complex64, device=hhat.device) * 1.0).contiguous()
    # keep the DC / Nyquist columns Hermitian so that the loss stays linear in the perturbation
    hs = base.hhat()
    fd = loss(w, hhat + dH, u) - loss(w, hhat - dH, u)
    an = 2 * torch.sum(dh.real.double() * dH.real.double() + dh.imag.double() * dH.imag.double()).item()
    assert abs(fd - an) <= 1e-3 * abs(an) + 1e-6
    dU = torch.randn_like(u) * 1.0
    fd = loss(w, hhat, u + dU) - loss(w, hhat, u - dU)
    an = 2 * torch.sum(du.double() * dU.double()).item()
    assert abs(fd - an) <= 1e-4 * abs(an)
    del hs


def test_backward_zero_batch(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    pr, r = _case((32, 32), 4, 1, 5)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    u = dev(torch, pr.u)[:0]
    du, dw, dh = plan.backward(u, u.clone())
    assert float(dw.abs().max()) == 0.0 and float(dh.abs().max()) == 0.0
