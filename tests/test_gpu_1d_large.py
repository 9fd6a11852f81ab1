"""GPU parity of 1D operators longer than 8192 points (the four-step path).

N = 2^14 .. 2^18 run as column FFTs, twiddles and row FFTs over an NY x NX
view of the sequence.  Checked against the FP64 oracle:
  - the plan's spectra hhat_k at sampled frequencies (oracle.dft.dft_at, the
    DFT definition evaluated one frequency at a time),
  - full forward and adjoint outputs for impulse responses of short support
    (the oracle's shift sum stays cheap), including odd m, m = 1 and batches
    that span two scratch chunks,
  - the periodised-Gaussian problem of Section 5 at N = 65536 on sampled
    outputs (gather form), plus the adjoint identity <H u, v> = <u, H* v>.
Bar: relative l2 <= 1e-5 (FP32 storage and arithmetic).
"""
import numpy as np
import pytest

import synth
from oracle import dft as D
from oracle import expansion as E

pytestmark = pytest.mark.gpu

TOL = 1e-5
SIZES = [1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18]


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


def rel_rows(got, ref):
    got = got.reshape(got.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def short_problem(n, m, batch, seed, radius=40):
    """Hat windows, random impulse responses supported on |offset| <= radius, N(0,1) input."""
    rng = np.random.default_rng(seed)
    w = synth.hat_windows_1d(n, m).astype(np.float32)
    h = np.zeros((m, n), np.float32)
    offs = np.arange(-radius, radius + 1) % n
    h[:, offs] = rng.standard_normal((m, offs.size)).astype(np.float32)
    u = rng.standard_normal((batch, n)).astype(np.float32)
    return w, h, u


@pytest.mark.parametrize("n", SIZES)
def test_large_1d_spectra_at_sampled_frequencies(torch_cuda, n):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    rng = np.random.default_rng(n)
    m = 3
    h = rng.standard_normal((m, n)).astype(np.float32)
    w = np.ones((m, n), np.float32)
    plan = Plan(dev(torch, w), h=dev(torch, h))
    got = plan.hhat().cpu().numpy().astype(np.complex128)
    assert got.shape == (m, n // 2 + 1)
    freqs = np.unique(np.concatenate([[0, 1, 2, n // 2 - 1, n // 2, n // 4, 127, 128, 129],
                                      rng.integers(0, n // 2 + 1, 48)]))
    ref = D.dft_at(h.astype(np.float64), freqs)
    ref[:, freqs == 0] = ref[:, freqs == 0].real
    ref[:, freqs == n // 2] = ref[:, freqs == n // 2].real
    err = np.linalg.norm(got[:, freqs] - ref) / np.linalg.norm(ref)
    assert err < 2e-6, err


@pytest.mark.parametrize("n,m,batch", [(1 << 14, 4, 2), (1 << 15, 3, 1), (1 << 16, 8, 2),
                                       (1 << 17, 5, 1), (1 << 18, 2, 1), (1 << 16, 1, 2)])
def test_large_1d_forward_adjoint_full_output(torch_cuda, n, m, batch):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    w, h, u = short_problem(n, m, batch, 300 + m)
    plan = Plan(dev(torch, w), h=dev(torch, h))
    ud = dev(torch, u)
    y = host(plan.apply(ud))
    x = host(plan.apply_adjoint(ud))
    assert rel_rows(y, E.apply(u, w, h)) < TOL
    assert rel_rows(x, E.apply_adjoint(u, w, h)) < TOL


def test_large_1d_batch_spans_scratch_chunks(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    n, m, batch = 1 << 14, 2, 70
    w, h, u = short_problem(n, m, batch, 41, radius=8)
    plan = Plan(dev(torch, w), h=dev(torch, h))
    ud = dev(torch, u)
    y = host(plan.apply(ud))
    x = host(plan.apply_adjoint(ud))
    assert rel_rows(y, E.apply(u, w, h)) < TOL
    assert rel_rows(x, E.apply_adjoint(u, w, h)) < TOL
    assert plan.apply(ud[:0]).shape == (0, n)


def test_large_1d_gaussian_problem_sampled_and_adjoint_identity(torch_cuda):
    """Periodised Gaussians sigma(y) = 0.01 + 0.005 sin(2 pi y) on hats, N = 65536, m = 8."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    n, m, batch = 1 << 16, 8, 2
    pr = synth.problem_1d(n, m, batch, 77)
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    ud = dev(torch, pr.u)
    y = host(plan.apply(ud))
    x = host(plan.apply_adjoint(ud))
    rng = np.random.default_rng(5)
    pts = np.unique(np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, 60)]))[:, None]
    ys = E.apply_at(pr.u, pr.w, pr.h, pts)
    xs = E.apply_adjoint_at(pr.u, pr.w, pr.h, pts)
    assert rel_rows(y[:, pts[:, 0]], ys) < TOL
    assert rel_rows(x[:, pts[:, 0]], xs) < TOL
    v = rng.standard_normal((batch, n)).astype(np.float32)
    hv = host(plan.apply_adjoint(dev(torch, v)))
    lhs = np.sum(y * v)
    rhs = np.sum(pr.u.astype(np.float64) * hv)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(y) * np.linalg.norm(v)


def test_large_1d_plan_from_spectra_round_trip(torch_cuda):
    """Plan built from exported spectra reproduces the original plan's applies."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    n, m = 1 << 15, 3
    w, h, u = short_problem(n, m, 2, 9)
    p1 = Plan(dev(torch, w), h=dev(torch, h))
    p2 = Plan(dev(torch, w), hhat=p1.hhat())
    ud = dev(torch, u)
    y1, y2 = host(p1.apply(ud)), host(p2.apply(ud))
    assert rel_rows(y2, y1) < 1e-6
    assert rel_rows(y2, E.apply(u, w, h)) < TOL


def test_large_1d_restrictions(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    from paper_1604_04374_gb300.pce import PceError
    n, m = 1 << 14, 2
    w, h, u = short_problem(n, m, 1, 3)
    with pytest.raises(PceError) as e:
        Plan(dev(torch, w), h=dev(torch, h), flags=pce.PCE_FLAG_LOWP_STORAGE)
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    plan = Plan(dev(torch, w), h=dev(torch, h))
    with pytest.raises(PceError) as e:
        plan.backward(dev(torch, u), dev(torch, u))
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    with pytest.raises(PceError) as e:
        pce.pce_plan_create(1, (1 << 19,), m, dev(torch, w).data_ptr(), dev(torch, h).data_ptr())
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED
