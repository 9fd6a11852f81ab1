"""GPU: sectioned applies (PCE_FLAG_SECTIONED, Lemma 3.2) against the FP64 oracle.

Every term is convolved on a 1024-row section sized to its window box plus
the support of h_k and added into the output; the operator is the same as the
whole-grid path's (the rounding order differs, and the atomic adds make it
vary from run to run), so both are checked against the oracle.
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


def short_h(pr, seed, ra=5, rb=3):
    """Random impulse responses supported on offsets [-ra, rb] x [-rb, ra] (asymmetric)."""
    rng = np.random.default_rng(seed)
    ny, nx = pr.shape
    h = np.zeros_like(pr.h)
    rows = np.arange(-ra, rb + 1) % ny
    cols = np.arange(-rb, ra + 1) % nx
    h[:, rows[:, None], cols[None, :]] = rng.standard_normal((pr.m, rows.size, cols.size)).astype(np.float32)
    return h


@pytest.mark.parametrize("ny,nx,m,batch", [(2048, 64, 64, 2), (1024, 128, 16, 1), (2048, 256, 64, 1),
                                            (1024, 1024, 16, 1)])
def test_sectioned_matches_oracle(torch_cuda, ny, nx, m, batch):
    """Section widths 32, 32, 128 and 1024."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(ny, nx, m, batch, 400 + m, "normal")
    h = short_h(pr, 7 + m)
    plan = Plan(dev(torch, pr.w), h=dev(torch, h), flags=pce.PCE_FLAG_SECTIONED)
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.apply(pr.u, pr.w, h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, h)) < TOL
    assert plan.launch_count(False, batch) == 3 and plan.launch_count(True, batch) == 3


def test_sectioned_with_psf_family_and_gradients(torch_cuda):
    """The anisotropic PSFs of the 2D workloads (their exact support is found at plan
    time); the gradients of a sectioned plan use its whole-grid structures."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(1024, 64, 16, 2, 431, "normal")
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_SECTIONED)
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL
    r = np.random.default_rng(3).standard_normal(pr.u.shape).astype(np.float32)
    du, dw, dh = plan.backward(u, dev(torch, r))
    rdu, rdw, _, rdh = E.grad(pr.u, pr.w, pr.h.astype(np.float64), r)
    assert rel(host(du), rdu) < TOL and rel(host(dw)[None], rdw[None]) < TOL


def test_sectioned_full_size_workload_sampled(torch_cuda):
    """2048 x 2048, m = 64, B = 4 (the reduced-storage workload's operator in FP32):
    sampled outputs against the oracle and agreement with the whole-grid path."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.workload("2d_2048_m64_b4")
    u = dev(torch, pr.u)
    sec = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_SECTIONED)
    gen = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    ys, xs = host(sec.apply(u)), host(sec.apply_adjoint(u))
    assert rel(ys, host(gen.apply(u))) < 2e-6
    assert rel(xs, host(gen.apply_adjoint(u))) < 2e-6
    rng = np.random.default_rng(4)
    pts = np.stack([rng.integers(0, 2048, 24), rng.integers(0, 2048, 24)], axis=-1)
    flat = pts[:, 0] * 2048 + pts[:, 1]
    assert rel(ys.reshape(4, -1)[:, flat], E.apply_at(pr.u, pr.w, pr.h, pts)) < TOL
    assert rel(xs.reshape(4, -1)[:, flat], E.apply_adjoint_at(pr.u, pr.w, pr.h, pts)) < TOL
    # every output of right-hand sides 0 and 3 against the compiled FP64 oracle:
    # all 192 sections, every column CTA and every row CTA of both directions
    from oracle import direct as C
    for b in (0, 3):
        yo = C.apply(pr.u[b:b + 1], pr.w, pr.h)
        xo = C.apply_adjoint(pr.u[b:b + 1], pr.w, pr.h)
        for got, ref in ((ys[b:b + 1], yo), (xs[b:b + 1], xo)):
            assert rel(got, ref) < TOL
            assert np.max(np.abs(got - ref)) < TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("ny,nx,m,batch", [(1024, 128, 16, 2), (2048, 256, 64, 1)])
def test_sectioned_reduced_storage_matches_oracle(torch_cuda, ny, nx, m, batch):
    """PCE_FLAG_SECTIONED | PCE_FLAG_LOWP_STORAGE: half2 section spectra with per-term
    scales and bfloat16 windows, FP32 arithmetic; against the FP64 oracle of the
    unrounded operator at the reduced-storage bar 3e-3, and against the FP32
    sectioned plan."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(ny, nx, m, batch, 450 + m, "normal")
    h = short_h(pr, 9 + m)
    w_d, h_d, u = dev(torch, pr.w), dev(torch, h), dev(torch, pr.u)
    low = Plan(w_d, h=h_d, flags=pce.PCE_FLAG_SECTIONED | pce.PCE_FLAG_LOWP_STORAGE)
    full = Plan(w_d, h=h_d, flags=pce.PCE_FLAG_SECTIONED)
    y, x = host(low.apply(u)), host(low.apply_adjoint(u))
    assert rel(y, E.apply(pr.u, pr.w, h)) < 3e-3
    assert rel(x, E.apply_adjoint(pr.u, pr.w, h)) < 3e-3
    assert rel(y, host(full.apply(u))) < 3e-3
    assert rel(x, host(full.apply_adjoint(u))) < 3e-3
    assert rel(y, host(full.apply(u))) > 1e-6   # the storage really is reduced


def test_sectioned_without_sections(torch_cuda):
    """Every h_k zero, or every w_k zero but one: no section for the dead terms; an
    operator without any section applies as zero."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(256, 64, 16, 2, 460, "normal")
    u = dev(torch, pr.u)
    zero = Plan(dev(torch, pr.w), h=dev(torch, np.zeros_like(pr.h)), flags=pce.PCE_FLAG_SECTIONED)
    assert float(zero.apply(u).abs().max()) == 0.0
    assert float(zero.apply_adjoint(u).abs().max()) == 0.0
    assert zero.launch_count(False, 2) == 0
    w1 = np.zeros_like(pr.w)
    w1[5] = pr.w[5]
    h = short_h(pr, 17)
    one = Plan(dev(torch, w1), h=dev(torch, h), flags=pce.PCE_FLAG_SECTIONED)
    assert rel(host(one.apply(u)), E.apply(pr.u, w1, h)) < TOL
    assert rel(host(one.apply_adjoint(u)), E.apply_adjoint(pr.u, w1, h)) < TOL


def test_sectioned_restrictions(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    from paper_1604_04374_gb300.pce import PceError
    pr = synth.problem_2d(1024, 64, 16, 1, 440, "normal")
    w, h = dev(torch, pr.w), dev(torch, pr.h)
    for flags in (pce.PCE_FLAG_SECTIONED | pce.PCE_FLAG_PRODUCT_CONVOLUTION,
                  pce.PCE_FLAG_SECTIONED | pce.PCE_FLAG_UNFUSED):
        with pytest.raises(PceError) as e:
            Plan(w, h=h, flags=flags)
        assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    hhat = torch.zeros((16, 1024, 33), dtype=torch.complex64, device="cuda")
    with pytest.raises(PceError) as e:
        Plan(w, hhat=hhat, flags=pce.PCE_FLAG_SECTIONED)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    # boxes of 1023 rows plus the PSF support do not fit a 1024-row section
    big = synth.problem_2d(2048, 32, 16, 1, 441, "normal")
    with pytest.raises(PceError) as e:
        Plan(dev(torch, big.w), h=dev(torch, big.h), flags=pce.PCE_FLAG_SECTIONED)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    w1 = dev(torch, np.ones((2, 256), np.float32))
    with pytest.raises(PceError) as e:
        Plan(w1, h=w1, flags=pce.PCE_FLAG_SECTIONED)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED


def test_sectioned_plan_in_a_batch_and_autotuned(torch_cuda):
    """A sectioned plan's forward and adjoint as two concurrent tasks of one batch graph
    (each lane has its own section scratch), and its autotune (one timed candidate)."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan, pce
    pr = synth.problem_2d(1024, 128, 16, 3, 470, "normal")
    h = short_h(pr, 19)
    plan = Plan(dev(torch, pr.w), h=dev(torch, h), flags=pce.PCE_FLAG_SECTIONED)
    chunk, variant, rvariant, ms = plan.autotune(3)
    assert ms > 0 and len(plan.tuning_log()) == 1
    u = dev(torch, pr.u)
    y, x = torch.empty_like(u), torch.empty_like(u)
    b = Batch([(plan, u, y, False), (plan, u, x, True)], lanes=2)
    for _ in range(2):   # a replay starts from the previous run's outputs
        b.launch()
        torch.cuda.synchronize()
        assert rel(host(y), E.apply(pr.u, pr.w, h)) < TOL
        assert rel(host(x), E.apply_adjoint(pr.u, pr.w, h)) < TOL
    b.close()


def test_sectioned_sections_wider_than_the_grid(torch_cuda):
    """A 15-column support on a 16-column grid: the work model takes sections of 32
    columns, wider than the grid, whose columns wrap by the remainder."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(256, 16, 4, 2, 480, "normal")
    h = short_h(pr, 21, ra=7, rb=7)
    plan = Plan(dev(torch, pr.w), h=dev(torch, h), flags=pce.PCE_FLAG_SECTIONED)
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.apply(pr.u, pr.w, h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, h)) < TOL


def test_sectioned_wavelet_windows(torch_cuda):
    """Wavelet windows (Section 4.3): boxes of several widths per plan and windows of
    both signs, cut into column tiles."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.wavelet_problem((256, 128), 2, 2, 2, 490)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_SECTIONED)
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_sectioned_separable_plan(torch_cuda):
    """pce_plan_create_separable with PCE_FLAG_SECTIONED: the tensor-product windows are
    expanded to w_k = wy_k (x) wx_k and applied by sections."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    wy, wx = synth.hat_factors_2d(1024, 128, 4, 4)
    w = np.einsum("kr,kc->krc", wy, wx).astype(np.float32)
    rng = np.random.default_rng(31)
    u = rng.standard_normal((2, 1024, 128)).astype(np.float32)
    pr = synth.Problem("sep", (1024, 128), 16, w, np.zeros_like(w), u)
    h = short_h(pr, 23)
    plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h), flags=pce.PCE_FLAG_SECTIONED)
    ud = dev(torch, u)
    assert rel(host(plan.apply(ud)), E.apply(u, w, h)) < TOL
    assert rel(host(plan.apply_adjoint(ud)), E.apply_adjoint(u, w, h)) < TOL
