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
