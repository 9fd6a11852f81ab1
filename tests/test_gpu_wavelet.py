"""GPU parity with the windows of the wavelet form (Section 4.3): periodic D4
scaling functions and wavelets of several scales, whose supports shrink from
most of the grid to 3 n / 2^j - 2 samples per axis, and which take both signs.
The plan's support boxes must follow each window; applies (both forms, FP32
and reduced storage, single and batched) must match the FP64 oracle.
"""
import numpy as np
import pytest

import synth
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


def cyclic_extent(flags):
    """Length of the shortest periodic interval holding every set flag."""
    n = len(flags)
    if not flags.any():
        return 0
    if flags.all():
        return n
    zeros = np.concatenate([~flags, ~flags])
    best = run = 0
    for z in zeros:
        run = run + 1 if z else 0
        best = max(best, min(run, n))
    return n - best


CASES = [((1024,), 2, 4, 2), ((4096,), 3, 3, 1), ((128, 128), 2, 2, 2), ((64, 256), 2, 2, 1),
         ((32, 1024), 2, 2, 1)]


@pytest.mark.parametrize("shape,j0,levels,batch", CASES)
def test_wavelet_windows_match_oracle(torch_cuda, shape, j0, levels, batch):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    pr = synth.wavelet_problem(shape, j0, levels, batch, 40 + levels)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    if len(shape) == 2:
        _, boxes, _ = plan.info()
        for k, (r0, nr, c0, nc) in enumerate(boxes):
            nzr = np.abs(pr.w[k]).max(axis=1) > 0
            nzc = np.abs(pr.w[k]).max(axis=0) > 0
            assert nr == cyclic_extent(nzr) and nc == cyclic_extent(nzc), k
        assert len({b[1] for b in boxes}) >= 2          # supports of several sizes
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_wavelet_windows_product_form_and_reduced_storage(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.wavelet_problem((128, 128), 2, 2, 2, 51)
    u = dev(torch, pr.u)
    p = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_PRODUCT_CONVOLUTION)
    assert rel(host(p.apply(u)), E.product_convolution(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(p.apply_adjoint(u)), E.product_convolution_adjoint(pr.u, pr.w, pr.h)) < TOL
    q = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_LOWP_STORAGE)
    assert rel(host(q.apply(u)), E.apply(pr.u, pr.w, pr.h)) < 3e-3
    assert rel(host(q.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < 3e-3


def test_wavelet_plans_in_a_tuned_batch(torch_cuda):
    """Plans with supports of many sizes, autotuned, run as one graph: outputs equal single applies."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan
    probs = [synth.wavelet_problem(s, 2, lv, 1, 60 + i)
             for i, (s, lv) in enumerate([((1024,), 4), ((64, 256), 2), ((128, 128), 1), ((32, 1024), 2)])]
    plans = [Plan(dev(torch, p.w), h=dev(torch, p.h)) for p in probs]
    for p in plans:
        p.autotune(1)
    ins = [dev(torch, p.u) for p in probs]
    refs = []
    for p, x in zip(plans, ins):
        refs.append((host(p.apply(x)), host(p.apply_adjoint(x))))
    outs = [(torch.empty_like(x), torch.empty_like(x)) for x in ins]
    tasks = []
    for p, x, (y, z) in zip(plans, ins, outs):
        tasks += [(p, x, y, False), (p, x, z, True)]
    b = Batch(tasks, lanes=4)
    b.launch()
    torch.cuda.synchronize()
    for (y, z), (ry, rz) in zip(outs, refs):
        assert np.array_equal(host(y), ry) and np.array_equal(host(z), rz)
    b.close()
