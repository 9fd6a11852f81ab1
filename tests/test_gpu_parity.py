"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar (relative l2 per right-hand side, FP32 storage and arithmetic): 1e-5.
Small cases are compared element by element over the whole output; the full
workload sizes are compared on sampled outputs that the oracle evaluates one
by one (gather form), plus the adjoint identity, which holds at any size.
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


def rel_l2(got, ref):
    got = got.reshape(got.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def plan_for(torch, pr):
    from paper_1604_04374_gb300 import Plan
    return Plan(dev(torch, pr.w), h=dev(torch, pr.h))


def run_both(torch, pr, plan=None):
    plan = plan or plan_for(torch, pr)
    u = dev(torch, pr.u)
    y = plan.apply(u)
    x = plan.apply_adjoint(u)
    torch.cuda.synchronize()
    return host(y), host(x)


def custom(shape, w, h, u, name="custom"):
    return synth.Problem(name, tuple(shape), w.shape[0], w.astype(np.float32), h.astype(np.float32),
                         u.astype(np.float32))


# --------------------------------------------------------------- FFT core

@pytest.mark.parametrize("shape", [(16,), (32,), (128,), (1024,), (4096,), (8192,),
                                   (16, 16), (32, 64), (64, 32), (256, 128), (16, 2048), (2048, 16),
                                   (512, 512)])
def test_plan_spectra_match_naive_dft(torch_cuda, shape):
    """hhat_k = R2C(h_k) computed by the library's FFT vs the oracle's naive DFT (O4)."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    rng = np.random.default_rng(len(shape) * 1000 + shape[-1])
    m = 3
    h = rng.standard_normal((m,) + shape).astype(np.float32)
    w = np.ones((m,) + shape, np.float32)
    plan = Plan(dev(torch, w), h=dev(torch, h))
    got = plan.hhat().cpu().numpy().astype(np.complex128)
    ref = np.stack([D.rdft_nd(h[k].astype(np.float64), len(shape)) for k in range(m)])
    if len(shape) == 2:
        # the plan keeps the Hermitian part of the DC and Nyquist columns (exact for real h)
        pass
    else:
        ref[:, 0] = ref[:, 0].real
        ref[:, -1] = ref[:, -1].real
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 2e-6, err


# ------------------------------------------------------------ small parity

SMALL_2D = [
    (16, 16, 4, 2), (64, 64, 4, 3), (32, 128, 8, 2), (128, 32, 8, 1), (64, 64, 16, 2),
    # a side of 1024 runs the one-warp FFT kernels (rows and columns)
    (16, 1024, 4, 2), (1024, 16, 4, 3), (32, 1024, 8, 1),
]


@pytest.mark.parametrize("ny,nx,m,batch", SMALL_2D)
def test_2d_forward_adjoint_full_output(torch_cuda, ny, nx, m, batch):
    pr = synth.problem_2d(ny, nx, m, batch, 100 + ny + nx + m, "normal")
    y, x = run_both(torch_cuda, pr)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


@pytest.mark.parametrize("n,m,batch", [(16, 3, 1), (64, 4, 3), (256, 8, 2), (1024, 8, 1), (1024, 5, 2),
                                       (2048, 16, 2), (4096, 8, 1), (8192, 4, 2), (512, 1, 1)])
def test_1d_forward_adjoint_full_output(torch_cuda, n, m, batch):
    pr = synth.problem_1d(n, m, batch, 200 + n + m)
    y, x = run_both(torch_cuda, pr)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_1d_workload_n1024_m8(torch_cuda):
    """1D N=1024, m=8 hats, periodised Gaussian sigma(y)=0.01+0.005 sin(2 pi y), B=1."""
    pr = synth.workload("1d_n1024_m8_b1")
    y, x = run_both(torch_cuda, pr)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


@pytest.mark.parametrize("shape", [(32, 64), (64, 16), (128,)])
def test_dense_random_windows_and_responses(torch_cuda, shape):
    """Full-support windows (no row skipping) and impulse responses with every tap nonzero."""
    rng = np.random.default_rng(7)
    m = 5
    w = rng.standard_normal((m,) + shape)
    h = rng.standard_normal((m,) + shape)
    u = rng.standard_normal((2,) + shape)
    pr = custom(shape, w, h, u)
    y, x = run_both(torch_cuda, pr)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


@pytest.mark.parametrize("shape", [(1024, 32), (16, 1024)])
def test_sparse_arbitrary_operator_at_1024(torch_cuda, shape):
    """Random windows on random boxes and random sparse impulse responses, one side 1024."""
    rng = np.random.default_rng(17)
    m = 3
    ny, nx = shape
    w = np.zeros((m,) + shape)
    for k in range(m):
        r0, c0 = rng.integers(0, ny), rng.integers(0, nx)
        nr, nc = rng.integers(1, ny + 1), rng.integers(1, nx + 1)
        rows = (r0 + np.arange(nr)) % ny
        cols = (c0 + np.arange(nc)) % nx
        w[k][np.ix_(rows, cols)] = rng.standard_normal((nr, nc))
    h = np.zeros((m,) + shape)
    idx = rng.integers(0, ny * nx, size=(m, 150))
    for k in range(m):
        h[k].reshape(-1)[idx[k]] = rng.standard_normal(150)
    u = rng.standard_normal((2,) + shape)
    pr = custom(shape, w, h, u)
    y, x = run_both(torch_cuda, pr)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_degenerate_windows(torch_cuda):
    """An all-zero window, a single-row window, a single-pixel window, windows across both seams."""
    torch = torch_cuda
    ny, nx = 64, 32
    rng = np.random.default_rng(8)
    m = 5
    w = np.zeros((m, ny, nx))
    w[1, 5, :] = rng.standard_normal(nx)                      # one row
    w[2, 63, 31] = 1.5                                         # one pixel at the corner
    w[3][np.ix_([62, 63, 0, 1, 2], [30, 31, 0, 1])] = rng.standard_normal((5, 4))   # both seams
    w[4, 10:41, 3:20] = rng.standard_normal((31, 17))          # odd box, 31 rows
    h = rng.standard_normal((m, ny, nx))
    u = rng.standard_normal((3, ny, nx))
    pr = custom((ny, nx), w, h, u)
    plan = plan_for(torch, pr)
    _, boxes, _ = plan.info()
    assert boxes[0][1] == 0
    assert boxes[1][:2] == (5, 1) and boxes[1][3] == nx
    assert boxes[2] == (63, 1, 31, 1)
    assert boxes[3] == (62, 5, 30, 4)
    assert boxes[4] == (10, 31, 3, 17)
    y, x = run_both(torch, pr, plan)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_pure_convolution_m1(torch_cuda):
    """m = 1, w = 1: a circular convolution (the FFT identity of Section 3.5)."""
    rng = np.random.default_rng(9)
    for shape in [(16, 16), (128, 256), (2048,)]:
        w = np.ones((1,) + shape)
        h = rng.standard_normal((1,) + shape)
        u = rng.standard_normal((2,) + shape)
        pr = custom(shape, w, h, u)
        y, x = run_both(torch_cuda, pr)
        axes = tuple(range(-len(shape), 0))
        ref = np.fft.irfftn(np.fft.rfftn(pr.h[0].astype(np.float64), axes=axes)
                            * np.fft.rfftn(pr.u.astype(np.float64), axes=axes), s=shape, axes=axes)
        assert rel_l2(y, ref) < TOL


# -------------------------------------------------------- from spectra

@pytest.mark.parametrize("shape", [(16, 32), (64,)])
def test_plan_from_spectra(torch_cuda, shape):
    """A plan from hhat (even a non-Hermitian one) is y = C2R(sum_k hhat_k . R2C(w_k u))."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    rng = np.random.default_rng(10)
    m = 3
    w = rng.standard_normal((m,) + shape).astype(np.float32)
    hs = (m,) + shape[:-1] + (shape[-1] // 2 + 1,)
    hhat = (rng.standard_normal(hs) + 1j * rng.standard_normal(hs)).astype(np.complex64)
    u = rng.standard_normal((2,) + shape).astype(np.float32)
    plan = Plan(dev(torch, w), hhat=dev(torch, hhat))
    y = host(plan.apply(dev(torch, u)))
    ref = E.apply_from_spectra(u, w, hhat.astype(np.complex128), shape)
    assert rel_l2(y, ref) < TOL
    # the adjoint is the transpose of that operator
    v = rng.standard_normal((2,) + shape).astype(np.float32)
    x = host(plan.apply_adjoint(dev(torch, v)))
    lhs = np.sum(ref * v)
    rhs = np.sum(u.astype(np.float64) * x)
    assert abs(lhs - rhs) < 1e-5 * np.sqrt(np.sum(ref ** 2) * np.sum(v.astype(np.float64) ** 2))


def test_plan_from_exported_spectra_matches(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    pr = synth.problem_2d(64, 128, 8, 2, 11)
    p1 = plan_for(torch, pr)
    p2 = Plan(dev(torch, pr.w), hhat=p1.hhat())
    u = dev(torch, pr.u)
    a = host(p1.apply(u))
    b = host(p2.apply(u))
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(a))


# ------------------------------------------- plain unfused comparator path

@pytest.mark.parametrize("ny,nx,m,batch", [(64, 64, 4, 3), (32, 128, 8, 2), (16, 16, 4, 1)])
def test_unfused_pipeline_matches_oracle(torch_cuda, ny, nx, m, batch):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    from paper_1604_04374_gb300.pce import PCE_FLAG_UNFUSED
    pr = synth.problem_2d(ny, nx, m, batch, 300 + ny + nx, "normal")
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=PCE_FLAG_UNFUSED)
    y, x = run_both(torch, pr, plan)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_unfused_pipeline_matches_fused_on_workload(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    from paper_1604_04374_gb300.pce import PCE_FLAG_UNFUSED
    pr = synth.workload("2d_1024_m16_b8")
    fused = plan_for(torch, pr)
    plain = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=PCE_FLAG_UNFUSED)
    u = dev(torch, pr.u)
    for direction in ("apply", "apply_adjoint"):
        a = host(getattr(fused, direction)(u))
        b = host(getattr(plain, direction)(u))
        assert rel_l2(a, b) < TOL
    assert plain.launch_count(False, 8) > fused.launch_count(False, 8)


# ------------------------------------------------------- workload sizes

def _sample_points(shape, count, seed):
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.integers(0, n, count) for n in shape], axis=-1)
    # include the seams and corners
    extra = np.array([[0, 0], [shape[0] - 1, shape[1] - 1], [0, shape[1] - 1], [shape[0] // 2, 0]])
    return np.concatenate([pts, extra[:, :len(shape)]])


@pytest.mark.parametrize("name", ["2d_1024_m16_b8", "2d_512_m16_b16", "2d_2048_m64_b4"])
def test_workload_sampled_parity_and_adjoint_identity(torch_cuda, name):
    torch = torch_cuda
    pr = synth.workload(name)
    plan = plan_for(torch, pr)
    u = dev(torch, pr.u)
    y = plan.apply(u)
    x = plan.apply_adjoint(u)
    torch.cuda.synchronize()
    pts = _sample_points(pr.shape, 300, 12)
    sel = (slice(None),) + tuple(pts.T)
    ys = host(y[sel])
    xs = host(x[sel])
    yr = E.apply_at(pr.u, pr.w, pr.h, pts)
    xr = E.apply_adjoint_at(pr.u, pr.w, pr.h, pts)
    assert rel_l2(ys, yr) < TOL
    assert rel_l2(xs, xr) < TOL
    # adjoint identity <H u, v> = <u, H* v> over the whole arrays (v = u rolled)
    v = torch.roll(u, shifts=(7, 3), dims=(-2, -1)).contiguous()
    hv = plan.apply_adjoint(v)
    lhs = torch.sum(y.double() * v.double()).item()
    rhs = torch.sum(u.double() * hv.double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_batch_chunks_and_zero_batch(torch_cuda):
    """Batches larger than one scratch chunk, and batch = 0."""
    torch = torch_cuda
    pr = synth.problem_2d(256, 256, 16, 3, 13)
    plan = plan_for(torch, pr)
    u = dev(torch, pr.u)
    y_all = host(plan.apply(u))
    for b in range(3):
        yb = host(plan.apply(u[b:b + 1].contiguous()))
        assert np.array_equal(yb[0], y_all[b])
    from paper_1604_04374_gb300 import pce_apply
    pce_apply(plan.handle, u.data_ptr(), u.data_ptr() + 4, 0, 0)   # batch 0: no-op, no check


def test_errors_are_reported(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import PceError, pce, pce_apply
    pr = synth.problem_2d(64, 64, 4, 1, 14)
    plan = plan_for(torch, pr)
    u = dev(torch, pr.u)
    with pytest.raises(PceError) as e:
        pce_apply(plan.handle, u.data_ptr(), u.data_ptr(), 1, 0)        # in place
    assert e.value.status == pce.PCE_ERR_INVALID
    cpu = torch.from_numpy(pr.u.copy())
    with pytest.raises(PceError) as e:
        pce_apply(plan.handle, cpu.data_ptr(), u.data_ptr(), 1, 0)      # host pointer
    assert e.value.status == pce.PCE_ERR_INVALID
    with pytest.raises(PceError) as e:
        pce.pce_plan_create(2, (64, 96), 4, u.data_ptr(), u.data_ptr())
    assert e.value.status == pce.PCE_ERR_UNSUPPORTED


def test_non_default_stream(torch_cuda):
    torch = torch_cuda
    pr = synth.problem_2d(128, 128, 4, 2, 15)
    plan = plan_for(torch, pr)
    u = dev(torch, pr.u)
    ref = host(plan.apply(u))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        y = plan.apply(u, stream=s)
    s.synchronize()
    assert np.array_equal(host(y), ref)


@pytest.mark.parametrize("ny,nx,m,batch", [(2048, 16, 4, 2), (2048, 64, 8, 1), (2048, 32, 16, 3)])
def test_2048_point_columns_two_warp_fft(torch_cuda, ny, nx, m, batch):
    """Columns of 2048: two warps per column (even / odd frequencies by decimation in
    frequency), forward and adjoint, FP32 and reduced storage, against the oracle."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(ny, nx, m, batch, 300 + m, "normal")
    y, x = run_both(torch, pr)
    assert rel_l2(y, E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(x, E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL
    lp = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_LOWP_STORAGE)
    u = dev(torch, pr.u)
    assert rel_l2(host(lp.apply(u)), E.apply(pr.u, pr.w, pr.h)) < 3e-3
    assert rel_l2(host(lp.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < 3e-3


def test_2048_point_columns_variants_agree(torch_cuda, tmp_path):
    """The block-Stockham column variant (forced through the tuning cache) and the
    product-convolution form on 2048-point columns."""
    torch = torch_cuda
    import json
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(2048, 32, 4, 2, 321, "normal")
    u = dev(torch, pr.u)
    p1 = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    cache = str(tmp_path / "t.jsonl")
    p1.autotune(2, cache)
    rec = json.loads(open(cache).read().splitlines()[0])
    with open(cache, "a") as f:
        f.write(json.dumps(dict(rec, variant=1 - rec["variant"])) + "\n")
    p2 = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    p2.autotune(2, cache)
    for fn, ref in (("apply", E.apply), ("apply_adjoint", E.apply_adjoint)):
        r = ref(pr.u, pr.w, pr.h)
        assert rel_l2(host(getattr(p1, fn)(u)), r) < TOL
        assert rel_l2(host(getattr(p2, fn)(u)), r) < TOL
    q = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_PRODUCT_CONVOLUTION)
    assert rel_l2(host(q.apply(u)), E.product_convolution(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(host(q.apply_adjoint(u)), E.product_convolution_adjoint(pr.u, pr.w, pr.h)) < TOL


@pytest.mark.parametrize("ny,nx,m,batch", [(512, 16, 4, 2), (512, 64, 8, 1), (512, 32, 16, 3)])
def test_512_point_columns_one_warp_fft(torch_cuda, ny, nx, m, batch):
    """Columns of 512: the one-warp 512-point FFT (16 values per lane, the last radix-2
    split over lane pairs) in column variant 0 and the block Stockham kernels in variant 1,
    forward and adjoint, FP32 and reduced storage, against the oracle; both variants
    agree to rounding."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    pr = synth.problem_2d(ny, nx, m, batch, 400 + m, "normal")
    u = dev(torch, pr.u)
    ry, rx = E.apply(pr.u, pr.w, pr.h), E.apply_adjoint(pr.u, pr.w, pr.h)
    outs = []
    for cv in (0, 1):
        plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
        plan.set_tuning(batch, cv, 0)
        y, x = host(plan.apply(u)), host(plan.apply_adjoint(u))
        assert rel_l2(y, ry) < TOL and rel_l2(x, rx) < TOL
        outs.append((y, x))
        plan.close()
    assert rel_l2(outs[0][0], outs[1][0]) < TOL and rel_l2(outs[0][1], outs[1][1]) < TOL
    lp = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_LOWP_STORAGE)
    assert rel_l2(host(lp.apply(u)), ry) < 3e-3
    assert rel_l2(host(lp.apply_adjoint(u)), rx) < 3e-3
    q = Plan(dev(torch, pr.w), h=dev(torch, pr.h), flags=pce.PCE_FLAG_PRODUCT_CONVOLUTION)
    assert rel_l2(host(q.apply(u)), E.product_convolution(pr.u, pr.w, pr.h)) < TOL
    assert rel_l2(host(q.apply_adjoint(u)), E.product_convolution_adjoint(pr.u, pr.w, pr.h)) < TOL
