"""GPU construction of (h_k, w_k) by L2 projection onto periodic hats
(pce_construct_projection_1d, Corollary 4.3) against the FP64 oracle, and the
constructed expansion fed to a plan.

The TVIR is the 1D workload's kernel: T[d][j] = g_sigma(y_j)(d / n) / n, the
periodised Gaussian with sigma(y) = 0.01 + 0.005 sin(2 pi y).
"""
import numpy as np
import pytest

import synth
from oracle import construct as C
from oracle import expansion as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_1604_04374_gb300 import build
    build.build()
    torch.cuda.init()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def tvir(n):
    """[n][n] float32: column j is the impulse response at y_j = j / n."""
    return np.stack([synth.gaussian_psf_1d(n, synth.sigma_1d(j / n)) for j in range(n)], axis=1).astype(np.float32)


@pytest.mark.parametrize("n,m", [(256, 8), (512, 16), (512, 5), (1024, 32)])
def test_projection_matches_oracle(torch_cuda, n, m):
    torch = torch_cuda
    from paper_1604_04374_gb300 import construct_projection_1d
    T = tvir(n)
    h, w = construct_projection_1d(dev(torch, T), m)
    h = h.cpu().numpy().astype(np.float64)
    w = w.cpu().numpy().astype(np.float64)
    B = C.hat_basis(n, m)
    assert np.abs(w - B.T).max() < 1e-6
    ref = C.projection_coefficients(T.astype(np.float64), m).T      # [m][n]
    assert np.linalg.norm(h - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("n,m,alpha", [(256, 8, 2), (512, 16, 3), (512, 5, 3), (1024, 32, 2), (256, 8, 1)])
def test_bspline_projection_matches_oracle(torch_cuda, n, m, alpha):
    """pce_construct_projection_bspline_1d (Corollary 4.3 on B_{alpha,m}) against the oracle:
    the B-spline windows and the projection coefficients."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import construct_projection_1d
    T = tvir(n)
    h, w = construct_projection_1d(dev(torch, T), m, alpha)
    h = h.cpu().numpy().astype(np.float64)
    w = w.cpu().numpy().astype(np.float64)
    assert np.abs(w - C.bspline_basis(n, m, alpha).T).max() < 1e-6
    ref = C.projection_coefficients(T.astype(np.float64), m, alpha).T
    assert np.linalg.norm(h - ref) / np.linalg.norm(ref) < 1e-5


def test_bspline_expansion_feeds_a_plan_and_beats_hats(torch_cuda):
    """The cubic-spline construction applied by a plan equals the oracle's expansion, and
    approximates the true operator better than the hat construction at the same m."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, construct_projection_1d
    n = 512
    T = tvir(n)
    u = np.random.default_rng(13).standard_normal((2, n)).astype(np.float32)
    idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % n
    K = T.astype(np.float64)[idx, np.arange(n)[None, :]]
    y_true = u.astype(np.float64) @ K.T
    err = {}
    for alpha in (1, 3):
        h, w = construct_projection_1d(dev(torch, T), 16, alpha)
        plan = Plan(w.contiguous(), h=h.contiguous())
        y = plan.apply(dev(torch, u)).cpu().numpy().astype(np.float64)
        ref = E.apply(u, w.cpu().numpy(), h.cpu().numpy())
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5
        err[alpha] = np.linalg.norm(y - y_true) / np.linalg.norm(y_true)
        plan.close()
    assert err[3] < err[1], err


def test_constructed_expansion_feeds_a_plan(torch_cuda):
    """Plan(w, h) from the construction applies sum_k h_k * (w_k . u); the error to the
    true operator u -> sum_j T[(i - j) mod n][j] u[j] does not grow over nested hat spaces."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, construct_projection_1d
    n = 512
    T = tvir(n)
    rng = np.random.default_rng(12)
    u = rng.standard_normal((2, n)).astype(np.float32)
    idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % n
    K = T.astype(np.float64)[idx, np.arange(n)[None, :]]                # K[i][j] = T[(i - j) mod n][j]
    y_true = u.astype(np.float64) @ K.T
    errs = []
    for m in (4, 8, 16, 32, 64):
        h, w = construct_projection_1d(dev(torch, T), m)
        plan = Plan(w.contiguous(), h=h.contiguous())
        y = plan.apply(dev(torch, u)).cpu().numpy().astype(np.float64)
        ref = E.apply(u, w.cpu().numpy(), h.cpu().numpy())
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5
        errs.append(np.linalg.norm(y - y_true) / np.linalg.norm(y_true))
    assert all(b <= a * (1 + 1e-3) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.2 * errs[0], errs


def test_projection_argument_errors(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import pce
    from paper_1604_04374_gb300.pce import PceError
    T = torch.zeros((64, 64), device="cuda")
    h = torch.empty((4, 64), device="cuda")
    with pytest.raises(PceError) as e:
        pce.pce_construct_projection_1d(T.data_ptr(), 64, 2, h.data_ptr(), h.data_ptr())
    assert e.value.status == pce.PCE_ERR_INVALID
    Tc = torch.zeros((64, 64))
    with pytest.raises(PceError) as e:
        pce.pce_construct_projection_1d(Tc.data_ptr(), 64, 4, h.data_ptr(), h.data_ptr())
    assert e.value.status == pce.PCE_ERR_INVALID
    for m, alpha in ((4, 3), (5, 0), (6, 4)):     # m < alpha + 2, orders outside 1..3
        with pytest.raises(PceError) as e:
            pce.pce_construct_projection_bspline_1d(T.data_ptr(), 64, m, alpha, h.data_ptr(), h.data_ptr())
        assert e.value.status == pce.PCE_ERR_INVALID


# ---------------------------------------------------------------- SVD (Section 5.1)

def fro_rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,m", [(256, 4), (256, 8), (1024, 12), (1024, 32)])
def test_svd_matches_oracle(torch_cuda, n, m):
    """Randomised SVD on the GPU against the oracle's exact SVD of the same float32
    TVIR: singular values, the rank-m approximation, the significant terms one by
    one (same sign rule), and orthonormal windows."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import construct_svd_1d
    T = tvir(n)
    h, w, s = construct_svd_1d(dev(torch, T), m)
    h, w, s = (t.cpu().numpy().astype(np.float64) for t in (h, w, s))
    rh, rw, rs = C.svd_terms(T.astype(np.float64), m)
    big = rs > 1e-4 * rs[0]
    assert np.abs(s[big] / rs[big] - 1).max() < 1e-5
    assert np.abs(s - rs).max() < 1e-6 * rs[0]
    assert fro_rel(h.T @ w, rh.T @ rw) < 1e-5
    for k in np.flatnonzero(big):
        assert fro_rel(w[k], rw[k]) < 1e-3 and fro_rel(h[k], rh[k]) < 1e-3
    assert np.abs(w @ w.T - np.eye(m)).max() < 1e-5
    # Eckart-Young: the residual is the tail of the spectrum
    tail = np.sqrt(np.sum(np.linalg.svd(T.astype(np.float64), compute_uv=False)[m:] ** 2))
    res = np.linalg.norm(T - h.T @ w)
    assert res <= tail + 1e-6 * np.linalg.norm(T)


def test_svd_rank_deficient_tvir(torch_cuda):
    """Example 3.3 (rank 2): the third and later terms come back as zeros."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import construct_svd_1d
    T = C.fig1_matrix(3).astype(np.float32)
    h, w, s = construct_svd_1d(dev(torch, T), 5)
    h, w, s = (t.cpu().numpy().astype(np.float64) for t in (h, w, s))
    rh, rw, rs = C.svd_terms(T.astype(np.float64), 2)
    assert np.abs(s[:2] / rs - 1).max() < 1e-5
    assert np.all(s[2:] == 0) and np.all(h[2:] == 0) and np.all(w[2:] == 0)
    assert fro_rel(h[:2].T @ w[:2], rh.T @ rw) < 1e-5


def test_svd_of_a_zero_tvir(torch_cuda):
    """T = 0 has no range: every term comes back as zeros, without an error."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import construct_svd_1d
    h, w, s = construct_svd_1d(torch.zeros((128, 128), device="cuda"), 6)
    assert float(h.abs().max()) == 0.0 and float(w.abs().max()) == 0.0 and float(s.abs().max()) == 0.0


def test_svd_expansion_feeds_a_plan(torch_cuda):
    """Plan(w, h) from the SVD (full-support windows) applies sum_k h_k * (w_k . u); its
    error to the true operator does not grow with m and reaches the float32 level."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, construct_svd_1d
    n = 512
    T = tvir(n)
    rng = np.random.default_rng(13)
    u = rng.standard_normal((2, n)).astype(np.float32)
    idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % n
    K = T.astype(np.float64)[idx, np.arange(n)[None, :]]
    y_true = u.astype(np.float64) @ K.T
    errs = []
    for m in (1, 2, 4, 8):
        h, w, _ = construct_svd_1d(dev(torch, T), m)
        plan = Plan(w.contiguous(), h=h.contiguous())
        y = plan.apply(dev(torch, u)).cpu().numpy().astype(np.float64)
        ref = E.apply(u, w.cpu().numpy(), h.cpu().numpy())
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5
        errs.append(np.linalg.norm(y - y_true) / np.linalg.norm(y_true))
    assert all(b <= a * (1 + 1e-3) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4, errs


def test_svd_argument_errors(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import pce
    from paper_1604_04374_gb300.pce import PceError
    T = torch.zeros((64, 64), device="cuda")
    h = torch.empty((4, 64), device="cuda")
    for n, m, p, q in ((64, 0, 10, 2), (64, 65, 0, 2), (64, 4, -1, 2), (64, 4, 10, 17), (8, 4, 0, 0)):
        with pytest.raises(PceError) as e:
            pce.pce_construct_svd_1d(T.data_ptr(), n, m, p, q, 0, h.data_ptr(), h.data_ptr())
        assert e.value.status == pce.PCE_ERR_INVALID
    Tc = torch.zeros((64, 64))
    with pytest.raises(PceError) as e:
        pce.pce_construct_svd_1d(Tc.data_ptr(), 64, 4, 10, 2, 0, h.data_ptr(), h.data_ptr())
    assert e.value.status == pce.PCE_ERR_INVALID


# ------------------------------------------------------- 2D projection (Corollary 4.3)

def tvir_2d_windowed(ny, nx, sy, sx, scale=0.6):
    """[ny][nx][sy][sx] float32: at every input position the workloads' anisotropic PSF
    (narrowed by `scale`) on the centred shift window."""
    T = np.zeros((ny, nx, sy, sx), dtype=np.float32)
    for r in range(ny):
        for c in range(nx):
            sxp, syp, th = synth.psf_params_2d(c / nx, r / ny)
            full = synth.aniso_psf_2d(ny, nx, scale * sxp, scale * syp, th)
            rows = (np.arange(sy) - sy // 2) % ny
            cols = (np.arange(sx) - sx // 2) % nx
            T[r, c] = full[np.ix_(rows, cols)].astype(np.float32)
    return T


def dense_from_windowed(T):
    """The [P][P] TVIR (shift d, input position j) the windowed form stands for."""
    ny, nx, sy, sx = T.shape
    P = ny * nx
    D = np.zeros((P, P))
    for r in range(ny):
        for c in range(nx):
            for a in range(sy):
                for b in range(sx):
                    d = ((a - sy // 2) % ny) * nx + (b - sx // 2) % nx
                    D[d, r * nx + c] += T[r, c, a, b]
    return D


@pytest.mark.parametrize("ny,nx,sy,sx,gy,gx", [(16, 24, 7, 9, 4, 3), (32, 32, 11, 11, 4, 4), (16, 16, 16, 16, 2, 2)])
def test_projection_2d_matches_oracle(torch_cuda, ny, nx, sy, sx, gy, gx):
    torch = torch_cuda
    from paper_1604_04374_gb300 import construct_projection_2d
    T = tvir_2d_windowed(ny, nx, sy, sx)
    h, wy, wx = construct_projection_2d(dev(torch, T), gy, gx)
    h, wy, wx = (t.cpu().numpy().astype(np.float64) for t in (h, wy, wx))
    B = C.tensor_hat_basis((ny, nx), gy, gx)                       # [P][m]
    np.testing.assert_allclose(np.einsum("kr,kc->krc", wy, wx).reshape(gy * gx, -1), B.T, atol=1e-6)
    ref = C.projection_coefficients_2d(dense_from_windowed(T), (ny, nx), gy, gx).T.reshape(gy * gx, ny, nx)
    assert np.linalg.norm(h - ref) / np.linalg.norm(ref) < 1e-5


def test_projection_2d_feeds_a_separable_plan(torch_cuda):
    """The construction's output applied by a separable plan equals the oracle's expansion,
    and the approximation of the true operator improves from a 2 x 2 to a 4 x 4 node grid."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, construct_projection_2d
    ny = nx = 32
    T = tvir_2d_windowed(ny, nx, 13, 13)
    D = dense_from_windowed(T)
    u = np.random.default_rng(14).standard_normal((2, ny, nx)).astype(np.float32)
    idx = np.indices((ny, nx)).reshape(2, -1).T
    P = ny * nx
    # the true operator: y[i] = sum_j T[(i - j) mod grid][j] u[j]
    K = np.zeros((P, P))
    for a, x in enumerate(idx):
        d = (x[None, :] - idx) % np.array([ny, nx])
        K[a] = D[d[:, 0] * nx + d[:, 1], np.arange(P)]
    y_true = u.reshape(2, -1).astype(np.float64) @ K.T
    errs = []
    for g in (2, 4):
        h, wy, wx = construct_projection_2d(dev(torch, T), g, g)
        plan = Plan(wy=wy.contiguous(), wx=wx.contiguous(), h=h.contiguous())
        y = plan.apply(dev(torch, u)).cpu().numpy().astype(np.float64)
        w = np.einsum("kr,kc->krc", wy.cpu().numpy(), wx.cpu().numpy())
        ref = E.apply(u, w, h.cpu().numpy())
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5
        errs.append(np.linalg.norm(y.reshape(2, -1) - y_true) / np.linalg.norm(y_true))
        plan.close()
    assert errs[1] < errs[0], errs


def test_projection_2d_argument_errors(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import pce
    from paper_1604_04374_gb300.pce import PceError
    T = torch.zeros((16, 16, 5, 5), device="cuda")
    h = torch.empty((16, 16, 16), device="cuda")
    w = torch.empty((16, 16), device="cuda")
    for args in ((16, 16, 5, 5, 1, 4), (16, 16, 5, 5, 4, 65), (16, 16, 0, 5, 4, 4), (16, 16, 17, 5, 4, 4),
                 (2, 16, 1, 5, 2, 2)):
        with pytest.raises(PceError) as e:
            pce.pce_construct_projection_2d(T.data_ptr(), *args, h.data_ptr(), w.data_ptr(), w.data_ptr())
        assert e.value.status == pce.PCE_ERR_INVALID
    with pytest.raises(PceError) as e:       # host memory
        Th = torch.zeros((16, 16, 5, 5))
        pce.pce_construct_projection_2d(Th.data_ptr(), 16, 16, 5, 5, 4, 4, h.data_ptr(), w.data_ptr(), w.data_ptr())
    assert e.value.status == pce.PCE_ERR_INVALID
