"""Pins for the seeded input generators: hat windows (Definition 2.2), periodised
Gaussian impulse responses (Poisson summation) and the rotated anisotropic PSF
(discrete moments equal the covariance)."""
import math

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("n,m", [(1024, 8), (64, 4), (96, 3)])
def test_hats_partition_of_unity_and_support(n, m):
    w = np.stack([synth.hat_1d(n, m, k) for k in range(m)])
    assert np.allclose(w.sum(axis=0), 1.0, atol=1e-15)
    for k in range(m):
        assert w[k].max() <= 1.0
        if n % m == 0:
            assert w[k][k * n // m] == 1.0
            # support 2/m: 2n/m - 1 nonzero samples (the ends are exact zeros)
            assert np.count_nonzero(w[k]) == 2 * n // m - 1
    wf = synth.hat_windows_1d(n, m)
    assert wf.dtype == np.float32
    assert np.allclose(wf.sum(axis=0), 1.0, atol=1e-6)


def test_2d_hats_tensor_product_and_node_grid():
    assert synth.node_grid(16) == (4, 4)
    assert synth.node_grid(8) == (4, 2)
    assert synth.node_grid(32) == (8, 4)
    assert synth.node_grid(4) == (2, 2)
    w = synth.hat_windows_2d(64, 32, 4, 2)
    assert w.shape == (8, 64, 32)
    assert np.allclose(w.sum(axis=0), 1.0, atol=1e-6)
    # node (a, c) = (1, 1) sits at row 16, col 16 with value 1
    assert w[1 * 2 + 1][16, 16] == 1.0


def test_gaussian_psf_1d_mass_and_symbol():
    n = 256
    for sigma in (0.005, 0.01, 0.015):
        h = synth.gaussian_psf_1d(n, sigma)
        # Poisson summation: sum_i h[i] = sum_l exp(-2 pi^2 sigma^2 (l n)^2) = 1 + tiny
        assert abs(h.sum() - 1.0) < 1e-13
        assert np.allclose(h[1:], h[1:][::-1], atol=1e-18)      # symmetric about 0


@pytest.mark.parametrize("sx,sy,th", [(1.5, 1.5, 0.0), (2.5, 1.5, 0.3), (1.6, 2.4, 2.0)])
def test_aniso_psf_moments_equal_covariance(sx, sy, th):
    h = synth.aniso_psf_2d(64, 64, sx, sy, th)
    assert abs(h.sum() - 1.0) < 1e-14
    d = np.arange(64)
    d = d - 64 * (d >= 32)
    X = d[None, :].astype(float)
    Y = d[:, None].astype(float)
    c, s = math.cos(th), math.sin(th)
    Sxx = c * c * sx ** 2 + s * s * sy ** 2
    Syy = s * s * sx ** 2 + c * c * sy ** 2
    Sxy = c * s * (sx ** 2 - sy ** 2)
    assert abs(np.sum(h * X * X) - Sxx) < 1e-10
    assert abs(np.sum(h * Y * Y) - Syy) < 1e-10
    assert abs(np.sum(h * X * Y) - Sxy) < 1e-10
    assert abs(np.sum(h * X)) < 1e-12 and abs(np.sum(h * Y)) < 1e-12


def test_workload_shapes_and_determinism():
    p = synth.problem_2d(64, 64, 4, 2, 5)
    q = synth.problem_2d(64, 64, 4, 2, 5)
    assert p.w.shape == (4, 64, 64) and p.h.shape == (4, 64, 64) and p.u.shape == (2, 64, 64)
    assert np.array_equal(p.u, q.u) and np.array_equal(p.h, q.h)
    assert p.u.dtype == np.float32
    r = synth.problem_1d(128, 8, 3, 0)
    assert r.w.shape == (8, 128) and r.u.shape == (3, 128)


def test_d4_filter_closed_form_properties():
    """Daubechies D4: sum sqrt(2), unit norm, orthogonal to its even shifts, two vanishing moments."""
    h = synth.D4_FILTER
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-15
    assert abs((h * h).sum() - 1.0) < 1e-15
    assert abs(h[0] * h[2] + h[1] * h[3]) < 1e-15
    g = np.array([(-1) ** i * h[3 - i] for i in range(4)])
    t = np.arange(4)
    assert abs(g.sum()) < 1e-15 and abs((t * g).sum()) < 1e-14


@pytest.mark.parametrize("n", [32, 128])
def test_periodic_wavelet_basis_is_orthonormal_and_complete(n):
    L = int(np.log2(n))
    funcs = [synth.periodic_wavelet(n, 2, k, "phi") for k in range(4)]
    for j in range(2, L):
        funcs += [synth.periodic_wavelet(n, j, k, "psi") for k in range(2 ** j)]
    B = np.stack(funcs)
    assert B.shape == (n, n)
    np.testing.assert_allclose(B @ B.T, np.eye(n), atol=1e-12)


def test_wavelet_window_supports_shrink_with_scale():
    """psi_{j,k} on n points is supported on 3 n / 2^j - 2 consecutive (periodic) samples."""
    n = 256
    for j in range(3, 8):
        for k in (0, 2 ** j - 1):
            f = synth.periodic_wavelet(n, j, k, "psi")
            assert np.count_nonzero(np.abs(f) > 1e-14) == 3 * n // 2 ** j - 2
    w, labels = synth.wavelet_windows_2d(32, 64, 2, 2)
    assert w.shape == (16 + 16 + 64, 32, 64) and len(labels) == w.shape[0]
    pr = synth.wavelet_problem((64,), 2, 3, 2, 9)
    assert pr.w.shape == (4 + 4 + 8 + 16, 64) and pr.u.shape == (2, 64)


@pytest.mark.parametrize("ny,nx,gy,gx", [(1024, 1024, 4, 4), (1024, 256, 2, 4), (64, 128, 8, 4)])
def test_hat_factors_reproduce_tensor_hats_exactly(ny, nx, gy, gx):
    wy, wx = synth.hat_factors_2d(ny, nx, gy, gx)
    w = synth.hat_windows_2d(ny, nx, gy, gx)
    assert np.array_equal(np.einsum("kr,kc->krc", wy, wx), w)
    assert np.array_equal((wy[:, :, None] * wx[:, None, :]).astype(np.float32), w)
