"""Pins for O1/O2/O3/O5: the expansion H_m u = sum_k h_k * (w_k . u) (Eq. 1.4) by definition.

Each pin is independent of the oracle's own formula: Lemma 3.1 (the TVIR of
the expansion is sum_k h_k(x) w_k(y)), the direct quadrature of a kernel that
is itself a rank-m convolution-product, the Poisson-summation closed form of
a periodised Gaussian, the library FFT, the adjoint identity and central
finite differences.
"""
import math

import numpy as np
import pytest

import synth
from oracle import dft as D
from oracle import expansion as E


def _rand_problem(shape, m, batch, seed, sparse=False):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((m,) + shape)
    h = rng.standard_normal((m,) + shape)
    if sparse:
        h[rng.random(h.shape) < 0.5] = 0.0
        w[rng.random(w.shape) < 0.3] = 0.0
    u = rng.standard_normal((batch,) + shape)
    return w, h, u


@pytest.mark.parametrize("shape", [(16,), (6, 10)])
def test_lemma_3_1_discrete_tvir_is_low_rank(shape):
    """Lemma 3.1: T_m(x, y) = sum_k h_k(x) w_k(y), with T(x, y) = K(x + y, y)."""
    m = 3
    w, h, _ = _rand_problem(shape, m, 1, 3)
    P = int(np.prod(shape))
    eye = np.eye(P).reshape((P,) + shape)
    K = E.apply(eye, w, h).reshape(P, P).T          # K[i, j] = (H_m e_j)[i]
    idx = np.indices(shape).reshape(len(shape), -1).T
    T = np.empty((P, P))
    for a, x in enumerate(idx):
        for b, y in enumerate(idx):
            xy = tuple((x + y) % np.array(shape))
            T[a, b] = K[np.ravel_multi_index(xy, shape), b]
    ref = sum(np.outer(h[k].reshape(-1), w[k].reshape(-1)) for k in range(m))
    assert np.max(np.abs(T - ref)) < 1e-12
    s = np.linalg.svd(T, compute_uv=False)
    assert s[m] < 1e-12 * s[0]


def test_lemma_3_1_quadrature_of_rank_m_kernel():
    """O3 of K(x, y) = sum_k h_k(x - y) w_k(y) equals O1 with h_k[i] = h_k(x_i)/N."""
    N, m = 64, 4
    sig = [0.03, 0.05, 0.02, 0.04]
    shift = [0.0, 0.05, -0.1, 0.2]

    def hfun(k, d):           # periodic, asymmetric impulse responses
        d = d - shift[k]
        d = d - np.floor(d + 0.5)
        return np.exp(-d ** 2 / (2 * sig[k] ** 2)) * (1 + 3 * d)

    def wfun(k, y):
        return np.cos(2 * np.pi * (k + 1) * y) + 0.5 * k

    def kernel(x, y):
        x = x[..., 0]
        y = y[..., 0]
        return sum(hfun(k, x - y) * wfun(k, y) for k in range(m))

    grid = np.arange(N) / N
    h = np.stack([hfun(k, grid) / N for k in range(m)])
    w = np.stack([wfun(k, grid) for k in range(m)])
    u = np.random.default_rng(4).standard_normal((2, N))
    y_quad = E.quadrature(kernel, u, (N,))
    y_exp = E.apply(u, w, h)
    assert np.max(np.abs(y_quad - y_exp)) < 1e-13 * np.max(np.abs(y_exp))


def test_pure_convolution_closed_form_1d():
    """m = 1, w = 1: a Fourier mode is multiplied by the Poisson-summation symbol.

    For h[i] = g_sigma(i/N)/N (periodised Gaussian), DFT(h)[f] = sum_l exp(-2 pi^2 sigma^2 (f + lN)^2).
    """
    N = 128
    sigma = 0.02
    h = synth.gaussian_psf_1d(N, sigma)[None]
    w = np.ones((1, N))
    j = np.arange(N)
    for f0 in (0, 1, 5, 17, 64):
        u = np.cos(2 * np.pi * f0 * j / N)[None]
        sym = sum(math.exp(-2 * math.pi ** 2 * sigma ** 2 * (f0 + l * N) ** 2) for l in range(-2, 3))
        y = E.apply(u, w, h)
        assert np.max(np.abs(y - sym * u)) < 1e-13


def test_pure_convolution_closed_form_2d_rotated_psf():
    """m = 1, w = 1 with the rotated anisotropic PSF: the symbol is
    exp(-2 pi^2 xi^T S xi), xi = (fx/Nx, fy/Ny), summed over aliases, over its value at 0."""
    ny, nx = 32, 64
    sx, sy, th = 1.9, 1.6, 0.7
    h = synth.aniso_psf_2d(ny, nx, sx, sy, th)[None]
    c, s = math.cos(th), math.sin(th)
    S = np.array([[c * c * sx ** 2 + s * s * sy ** 2, c * s * (sx ** 2 - sy ** 2)],
                  [c * s * (sx ** 2 - sy ** 2), s * s * sx ** 2 + c * c * sy ** 2]])

    def sym(fx, fy):
        tot = 0.0
        for lx in (-1, 0, 1):
            for ly in (-1, 0, 1):
                xi = np.array([fx / nx + lx, fy / ny + ly])
                tot += math.exp(-2 * math.pi ** 2 * xi @ S @ xi)
        return tot

    norm = sym(0, 0)
    rows, cols = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    w = np.ones((1, ny, nx))
    for fx, fy in [(1, 0), (0, 1), (3, 2), (3, -2), (-5, 7), (20, 9)]:
        u = np.cos(2 * np.pi * (fx * cols / nx + fy * rows / ny))[None]
        y = E.apply(u, w, h)
        assert np.max(np.abs(y - sym(fx, fy) / norm * u)) < 1e-12


@pytest.mark.parametrize("shape", [(32,), (8, 16), (16, 8)])
def test_fft_identity_library_and_naive(shape):
    """Section 3.5: each term equals C2R(R2C(h_k) . R2C(w_k u)) (library FFT and O4)."""
    m = 3
    w, h, u = _rand_problem(shape, m, 2, 5, sparse=True)
    y = E.apply(u, w, h)
    axes = tuple(range(-len(shape), 0))
    ref = sum(np.fft.irfftn(np.fft.rfftn(h[k], axes=axes) * np.fft.rfftn(w[k] * u, axes=axes),
                            s=shape, axes=axes) for k in range(m))
    assert np.max(np.abs(y - ref)) < 1e-12
    hhat = np.stack([D.rdft_nd(h[k], len(shape)) for k in range(m)])
    y2 = E.apply_from_spectra(u, w, hhat, shape)
    assert np.max(np.abs(y - y2)) < 1e-12


@pytest.mark.parametrize("shape", [(32,), (8, 16)])
def test_adjoint_identity_and_transpose(shape):
    m = 4
    w, h, u = _rand_problem(shape, m, 3, 6, sparse=True)
    v = np.random.default_rng(7).standard_normal(u.shape)
    lhs = np.sum(E.apply(u, w, h) * v)
    rhs = np.sum(u * E.apply_adjoint(v, w, h))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)
    P = int(np.prod(shape))
    eye = np.eye(P).reshape((P,) + shape)
    A = E.apply(eye, w, h).reshape(P, P)
    At = E.apply_adjoint(eye, w, h).reshape(P, P)
    assert np.max(np.abs(A - At.T)) < 1e-12


@pytest.mark.parametrize("shape", [(64,), (16, 32)])
def test_sampled_forms_match_full(shape):
    m = 3
    w, h, u = _rand_problem(shape, m, 2, 8, sparse=True)
    rng = np.random.default_rng(9)
    pts = np.stack([rng.integers(0, n, 20) for n in shape], axis=-1)
    y = E.apply(u, w, h)
    x = E.apply_adjoint(u, w, h)
    ys = E.apply_at(u, w, h, pts)
    xs = E.apply_adjoint_at(u, w, h, pts)
    sel = (slice(None),) + tuple(pts.T)
    assert np.max(np.abs(ys - y[sel])) < 1e-12
    assert np.max(np.abs(xs - x[sel])) < 1e-12


def _fd(fun, p, d, eps=1e-3):
    return (fun(p + eps * d) - fun(p - eps * d)) / (2 * eps)


@pytest.mark.parametrize("shape", [(16,), (8, 16), (64, 64)])
def test_gradients_central_fd(shape):
    """O5 against central finite differences (step 1e-3; the loss is linear in each argument)."""
    m = 4 if len(shape) == 2 else 3
    w, h, u = _rand_problem(shape, m, 2, 10)
    if shape == (64, 64):
        # the PSF family and hats of the 2D workloads, at 64x64 with m = 4
        pr = synth.problem_2d(64, 64, 4, 2, 99, "uniform", (2, 2))
        w, h, u = (pr.w.astype(np.float64), pr.h.astype(np.float64), pr.u.astype(np.float64))
        h[np.abs(h) < 1e-12] = 0.0
    rng = np.random.default_rng(11)
    r = rng.standard_normal(u.shape)
    du, dw, dh, dhh = E.grad(u, w, h, r)
    L = lambda uu, ww, hh: np.sum(E.apply(uu, ww, hh) * r)
    for name, g, fun, p in [("u", du, lambda q: L(q, w, h), u),
                            ("w", dw, lambda q: L(u, q, h), w),
                            ("h", dh, lambda q: L(u, w, q), h)]:
        for trial in range(2):
            d = rng.standard_normal(p.shape)
            if name == "h":
                d = d * (h != 0)           # stay on the tap support used by the shift sum
            fd = _fd(fun, p, d)
            an = np.sum(g * d)
            assert abs(fd - an) < 1e-9 * (abs(an) + np.sqrt(np.sum(g * g))), name
    hhat = np.stack([D.rdft_nd(h[k], len(shape)) for k in range(m)])
    Ls = lambda q: np.sum(E.apply_from_spectra(u, w, q, shape) * r)
    for trial in range(2):
        d = rng.standard_normal(hhat.shape) + 1j * rng.standard_normal(hhat.shape)
        fd = _fd(Ls, hhat, d)
        an = np.sum(dhh.real * d.real + dhh.imag * d.imag)
        assert abs(fd - an) < 1e-9 * (abs(an) + np.sqrt(np.sum(np.abs(dhh) ** 2)))
    # C2R discards Im of the DC/Nyquist bins of the last axis: their gradient is zero.
    nx = shape[-1]
    if len(shape) == 1:
        scale = np.max(np.abs(dhh))
        assert np.max(np.abs(dhh[..., 0].imag)) < 1e-14 * scale
        assert np.max(np.abs(dhh[..., nx // 2].imag)) < 1e-14 * scale


def _dense_product_convolution(w, h):
    """Matrix of u -> sum_k w_k(x) h_k(x - y) u(y) built entry by entry from the kernel
    formula of the product-convolution form (Section 1), not from the shift sum."""
    shape = w.shape[1:]
    P = int(np.prod(shape))
    idx = [np.unravel_index(i, shape) for i in range(P)]
    K = np.zeros((P, P))
    for a, xi in enumerate(idx):
        for b, yi in enumerate(idx):
            d = tuple((xi[t] - yi[t]) % shape[t] for t in range(len(shape)))
            K[a, b] = sum(w[k][xi] * h[k][d] for k in range(w.shape[0]))
    return K


@pytest.mark.parametrize("shape", [(12,), (4, 6)])
def test_product_convolution_matches_kernel_matrix(shape):
    """O6 and its adjoint against the dense kernel K(x, y) = sum_k w_k(x) h_k(x - y) and its transpose."""
    rng = np.random.default_rng(31)
    m = 3
    w = rng.standard_normal((m,) + shape)
    h = rng.standard_normal((m,) + shape)
    u = rng.standard_normal((2,) + shape)
    K = _dense_product_convolution(w, h)
    P = int(np.prod(shape))
    got = E.product_convolution(u, w, h).reshape(2, P)
    np.testing.assert_allclose(got, u.reshape(2, P) @ K.T, rtol=1e-12, atol=1e-12)
    got = E.product_convolution_adjoint(u, w, h).reshape(2, P)
    np.testing.assert_allclose(got, u.reshape(2, P) @ K, rtol=1e-12, atol=1e-12)


def test_product_convolution_special_cases():
    """Constant windows commute with the convolution (both forms agree); a single
    delta h_k = delta_0 gives the pointwise product (sum_k w_k) . u."""
    rng = np.random.default_rng(32)
    shape = (16, 8)
    m = 4
    c = rng.standard_normal(m)
    w = np.ones((m,) + shape) * c[:, None, None]
    h = rng.standard_normal((m,) + shape)
    u = rng.standard_normal((2,) + shape)
    np.testing.assert_allclose(E.product_convolution(u, w, h), E.apply(u, w, h), rtol=1e-12, atol=1e-12)
    w = rng.standard_normal((m,) + shape)
    h = np.zeros((m,) + shape)
    h[:, 0, 0] = 1.0
    np.testing.assert_allclose(E.product_convolution(u, w, h), w.sum(axis=0) * u, rtol=1e-13, atol=1e-13)
    v = rng.standard_normal((2,) + shape)
    h = rng.standard_normal((m,) + shape)
    lhs = np.sum(E.product_convolution(u, w, h) * v)
    rhs = np.sum(u * E.product_convolution_adjoint(v, w, h))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
