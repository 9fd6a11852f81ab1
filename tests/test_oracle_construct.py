"""Pins for the oracle's constructions: Fig. 1 (values printed in the paper), Example 3.3's
rank, nested hat projections (Corollary 4.3), interpolation on hats (Section 4), and the
Eckart-Young identity of the SVD construction (Section 5.1)."""
import os

import numpy as np
import pytest

import synth
from oracle import construct as C
from oracle import expansion as E

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(example):
    vals = np.loadtxt(os.path.join(GOLDEN, f"fig1_spectrum_{example}.txt"), comments="#")
    return vals[:, 1]


@pytest.mark.parametrize("example,count,tol", [(1, 10, 1e-10), (2, 10, 1e-13), (3, 2, 1e-11)])
def test_fig1_singular_values(example, count, tol):
    """Fig. 1: the leading singular values of J printed in the paper."""
    ref = _golden(example)
    s = C.fig1_singular_values(example)
    rel = np.abs(s[:count] / ref[:count] - 1.0)
    assert np.max(rel) < tol, rel


def test_fig1_whole_curves_agree_above_rounding():
    # Every printed value above the rounding floor (1e-13 of the first) is reproduced
    # to 1e-6 relative, up to an absolute SVD rounding error of 1e-16 of the first.
    for ex in (1, 2, 3):
        ref = _golden(ex)
        s = C.fig1_singular_values(ex)
        big = ref > 1e-13 * ref[0]
        err = np.abs(s[big] - ref[big])
        assert np.all(err <= 1e-6 * ref[big] + 1e-16 * ref[0]), np.max(err / ref[big])


def test_example_3_3_has_rank_two():
    s = C.fig1_singular_values(3)
    assert s[2] < 1e-13 * s[0]
    assert s[1] > 0.1 * s[0]


def test_projection_error_non_increasing_on_nested_hat_spaces():
    """Corollary 4.3: nested hat spaces (dyadic m) give a non-increasing L2 error, rate m^-2."""
    n = 512
    t = np.arange(n) / n
    x = t - np.floor(t + 0.5)
    s = 0.08 + 0.02 * np.cos(2 * np.pi * t)
    T = np.exp(-(x[:, None] ** 2) / (2 * s[None, :] ** 2))     # T(x_i, y_j), periodic in y
    errs = [np.linalg.norm(T - C.project_on_hats(T, m)) for m in (4, 8, 16, 32, 64)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:])), errs
    slope = np.log(errs[-1] / errs[-2]) / np.log(2)
    assert -2.3 < slope < -1.7, slope
    # the projection never loses to interpolation on the same space
    for m in (8, 32):
        assert (np.linalg.norm(T - C.project_on_hats(T, m))
                <= np.linalg.norm(T - C.interpolate_on_hats(T, m)) * (1 + 1e-12))


def test_interpolation_is_cardinal_and_exact_at_nodes():
    n, m = 64, 8
    B = C.hat_basis(n, m)
    nodes = np.arange(m) * n // m
    assert np.array_equal(B[nodes], np.eye(m))
    assert np.allclose(B.sum(axis=1), 1.0, atol=1e-15)
    T = np.random.default_rng(0).standard_normal((16, n))
    Tm = C.interpolate_on_hats(T, m)
    assert np.allclose(Tm[:, nodes], T[:, nodes], atol=1e-14)


def test_svd_truncation_error_is_tail_of_spectrum():
    T = C.fig1_matrix(1, 128)
    s = np.linalg.svd(T, compute_uv=False)
    for m in (1, 3, 6):
        err = np.linalg.norm(T - C.svd_truncate(T, m))
        assert abs(err - np.sqrt(np.sum(s[m:] ** 2))) < 1e-12 * s[0]


def test_interpolated_expansion_error_decreases_with_m():
    """H_m built like the 1D workload (hats at k/m, h_k = T(., y_k)) approaches the
    quadrature of the true kernel K(x, y) = g_sigma(y)(x - y) as m grows (O1 vs O3)."""
    N = 256

    def kernel(x, y):
        x = x[..., 0]
        y = y[..., 0]
        s = 0.01 + 0.005 * np.sin(2 * np.pi * y)
        d = x - y
        d = d - np.floor(d + 0.5)
        g = 0.0
        for j in (-1.0, 0.0, 1.0):
            g = g + np.exp(-((d + j) ** 2) / (2 * s ** 2))
        return g / (np.sqrt(2 * np.pi) * s)

    eye = np.eye(N)
    Hq = E.quadrature(kernel, eye, (N,))                       # rows: H e_j
    errs = []
    for m in (4, 8, 16, 32, 64):
        w = synth.hat_windows_1d(N, m).astype(np.float64)
        h = np.stack([synth.gaussian_psf_1d(N, synth.sigma_1d(k / m)) for k in range(m)])
        Hm = E.apply(eye, w, h)
        errs.append(np.linalg.norm(Hq - Hm) / np.linalg.norm(Hq))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    slope = np.log(errs[-1] / errs[-2]) / np.log(2)
    assert -2.4 < slope < -1.6, (errs, slope)


def test_projection_coefficients_reproduce_rows_in_the_hat_span():
    """Idempotence: rows that already are combinations of the hats come back exactly,
    and the residual of a general T is orthogonal to every hat (normal equations)."""
    rng = np.random.default_rng(8)
    n, m = 96, 12
    B = C.hat_basis(n, m)
    C0 = rng.standard_normal((n, m))
    np.testing.assert_allclose(C.projection_coefficients(C0 @ B.T, m), C0, atol=1e-10)
    T = rng.standard_normal((n, n))
    R = T - C.projection_coefficients(T, m) @ B.T
    assert np.abs(R @ B).max() < 1e-10 * np.abs(T).max() * n


def test_svd_terms_reproduce_the_printed_spectra_and_are_orthonormal():
    """The singular values of svd_terms on the Fig. 1 matrices are the printed
    ones (first values, with the global factors of the Fig. 1 readings); the
    windows are orthonormal and the responses orthogonal with norms sigma_k."""
    for ex in (1, 2):
        gold = _golden(ex)
        h, w, s = C.svd_terms(C.fig1_matrix(ex), 8)
        assert np.allclose(s * C.FIG1_SCALE[ex], gold[:8], rtol=1e-9, atol=0)
        assert np.allclose(w @ w.T, np.eye(8), atol=1e-12)
        assert np.allclose(h @ h.T, np.diag(s ** 2), atol=1e-12 * s[0] ** 2)
        assert np.all(w.sum(axis=1) >= 0)


def test_svd_terms_closed_forms():
    """A rank-one TVIR a b^t gives h_0 = |b| a, w_0 = b / |b| (sum of b positive);
    Example 3.3 has rank 2, so every further term is zero (Section 3)."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal(32)
    b = rng.random(32) + 0.1
    h, w, s = C.svd_terms(np.outer(a, b), 3)
    assert np.allclose(h[0], np.linalg.norm(b) * a, atol=1e-12)
    assert np.allclose(w[0], b / np.linalg.norm(b), atol=1e-14)
    assert np.all(h[1:] == 0) and np.all(w[1:] == 0)
    h, w, s = C.svd_terms(C.fig1_matrix(3), 5)
    assert s[1] > 0.1 and np.all(s[2:] == 0) and np.all(h[2:] == 0)


def test_svd_expansion_is_exact_for_a_rank_m_kernel():
    """Lemma 3.1: a kernel K(x, y) = sum_k h_k(x - y) w_k(y) of rank m is
    reproduced exactly by the m SVD terms of its TVIR, applied as Eq. 1.4
    (expansion.apply against the dense matrix built entry by entry)."""
    n, m = 48, 3
    rng = np.random.default_rng(8)
    h0 = rng.standard_normal((m, n))
    w0 = rng.standard_normal((m, n))
    T = h0.T @ w0                                   # T[d][j] = sum_k h_k[d] w_k[j]
    h, w, s = C.svd_terms(T, m)
    K = np.array([[T[(i - j) % n, j] for j in range(n)] for i in range(n)])
    u = rng.standard_normal((2, n))
    assert np.allclose(E.apply(u, w, h), u @ K.T, atol=1e-11)


@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_bspline_closed_forms_follow_the_definition(alpha):
    """Definition 2.2: B_{alpha,m} = m B_{0,m} * B_{alpha-1,m}, B_{0,m} the indicator of
    [-1/(2m), 1/(2m)].  The recursion, evaluated by numerical convolution from the
    indicator up (on unit knot spacing, m = 1), matches the piecewise polynomials; the
    B-splines are even, supported on |u| < (alpha + 1) / 2, and their translates by the
    nodes sum to one."""
    h = 1e-4
    s = np.arange(-0.5 + h / 2, 0.5, h)                     # midpoint rule over B_0's support
    u = np.linspace(-3.0, 3.0, 241)
    prev = lambda v: (np.abs(v) <= 0.5).astype(float)      # noqa: E731
    for a in range(1, alpha + 1):
        cur_vals = np.array([np.sum(prev(x - s)) * h for x in u])
        prev_tab = (u.copy(), cur_vals)
        prev = lambda v, t=prev_tab: np.interp(v, t[0], t[1], left=0.0, right=0.0)  # noqa: E731
    np.testing.assert_allclose(C.cardinal_bspline(alpha, u), cur_vals, atol=5e-3 if alpha == 1 else 2e-3)
    assert np.all(C.cardinal_bspline(alpha, u[np.abs(u) >= (alpha + 1) / 2]) == 0)
    np.testing.assert_array_equal(C.cardinal_bspline(alpha, u), C.cardinal_bspline(alpha, -u))
    B = C.bspline_basis(384, 12, alpha)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
    if alpha == 1:
        np.testing.assert_array_equal(B, C.hat_basis(384, 12))


@pytest.mark.parametrize("alpha", [2, 3])
def test_bspline_projection_idempotent_and_orthogonal(alpha):
    """Corollary 4.3 on B_{alpha,m}: rows already in the span come back exactly, and the
    residual of a general T is orthogonal to every B-spline (normal equations)."""
    rng = np.random.default_rng(9 + alpha)
    n, m = 120, 10
    B = C.bspline_basis(n, m, alpha)
    C0 = rng.standard_normal((n, m))
    np.testing.assert_allclose(C.projection_coefficients(C0 @ B.T, m, alpha), C0, atol=1e-9)
    T = rng.standard_normal((n, n))
    R = T - C.projection_coefficients(T, m, alpha) @ B.T
    assert np.abs(R @ B).max() < 1e-10 * np.abs(T).max() * n


def test_bspline_projection_rates_and_nesting():
    """Corollary 4.3: for a smooth TVIR the projection error falls like m^-(alpha + 1)
    for splines of degree alpha.  Odd orders have knots at multiples of 1/m, so the
    dyadic spaces are nested and the error cannot increase; the cubic space beats the
    hat space at every m."""
    n = 1024
    t = np.arange(n) / n
    x = t - np.floor(t + 0.5)
    s = 0.08 + 0.02 * np.cos(2 * np.pi * t)
    T = np.exp(-(x[:, None] ** 2) / (2 * s[None, :] ** 2))
    ms = (8, 16, 32, 64)
    for alpha in (1, 2, 3):
        errs = [np.linalg.norm(T - C.project_on_bsplines(T, m, alpha)) for m in ms]
        slope = np.log(errs[-1] / errs[-2]) / np.log(2)
        assert -(alpha + 1) - 0.4 < slope < -(alpha + 1) + 0.4, (alpha, slope)
        if alpha % 2 == 1:
            assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:])), (alpha, errs)
    for m in ms:
        assert (np.linalg.norm(T - C.project_on_bsplines(T, m, 3))
                < np.linalg.norm(T - C.project_on_bsplines(T, m, 1)))


def _tvir_2d(shape, seed):
    """A smooth space-varying 2D TVIR T[d][j] (shift d, input position j, flattened):
    the anisotropic PSF family of the workloads evaluated at every input position."""
    ny, nx = shape
    P = ny * nx
    T = np.zeros((P, P))
    for r in range(ny):
        for c in range(nx):
            sx, sy, th = synth.psf_params_2d(c / nx, r / ny)
            T[:, r * nx + c] = synth.aniso_psf_2d(ny, nx, 0.6 * sx, 0.6 * sy, th).reshape(-1)
    return T


def test_tensor_hat_projection_idempotent_orthogonal_and_separable():
    """Corollary 4.3 with 2D tensor-product hats: rows in the span come back exactly, the
    residual is orthogonal to every window, and the Gram matrix factors as the Kronecker
    product of the 1D ones (the windows are products of 1D hats), so that a TVIR that is a
    product of 1D TVIRs has the product of the 1D projections."""
    shape, gy, gx = (12, 16), 3, 4
    P = 12 * 16
    B = C.tensor_hat_basis(shape, gy, gx)
    assert B.shape == (P, gy * gx)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)       # partition of unity
    rng = np.random.default_rng(17)
    C0 = rng.standard_normal((P, gy * gx))
    np.testing.assert_allclose(C.projection_coefficients_2d(C0 @ B.T, shape, gy, gx), C0, atol=1e-9)
    T = rng.standard_normal((P, P))
    R = T - C.projection_coefficients_2d(T, shape, gy, gx) @ B.T
    assert np.abs(R @ B).max() < 1e-10 * np.abs(T).max() * P
    by, bx = C.hat_basis(12, gy), C.hat_basis(16, gx)
    np.testing.assert_allclose(B.T @ B, np.kron(by.T @ by, bx.T @ bx), atol=1e-12)
    # product TVIR: T[(a,b)][(r,c)] = Ty[a][r] Tx[b][c] -> coefficients are products
    Ty, Tx = rng.standard_normal((12, 12)), rng.standard_normal((16, 16))
    Tp = np.einsum("ar,bc->abrc", Ty, Tx).reshape(P, P)
    cp = C.projection_coefficients_2d(Tp, shape, gy, gx)
    ref = np.einsum("ai,bl->abil", C.projection_coefficients(Ty, gy), C.projection_coefficients(Tx, gx)).reshape(P, -1)
    np.testing.assert_allclose(cp, ref, atol=1e-10)


def test_tensor_hat_projection_error_falls_on_refined_node_grids():
    """Nested node grids (2 x 2 -> 4 x 4 -> 8 x 8 on a 32 x 32 grid) give non-increasing
    projection errors (nested subspaces), and the expansion built from the coefficients
    applies the projected operator through Eq. 1.4."""
    shape = (32, 32)
    T = _tvir_2d(shape, 0)
    errs = []
    for g in (2, 4, 8):
        B = C.tensor_hat_basis(shape, g, g)
        Tm = C.projection_coefficients_2d(T, shape, g, g) @ B.T
        errs.append(np.linalg.norm(T - Tm))
    assert errs[1] <= errs[0] * (1 + 1e-12) and errs[2] <= errs[1] * (1 + 1e-12), errs
    assert errs[2] < 0.5 * errs[0], errs
    # Lemma 3.1 on the grid: h_k = coefficient column k (over shifts), w_k = window k
    g = 4
    Cf = C.projection_coefficients_2d(T, shape, g, g)
    B = C.tensor_hat_basis(shape, g, g)
    h = Cf.T.reshape(g * g, *shape)
    w = B.T.reshape(g * g, *shape)
    u = np.random.default_rng(3).standard_normal((1,) + shape)
    Tm = Cf @ B.T                                            # Tm[d][j]
    idx = np.indices(shape).reshape(2, -1).T
    # y[i] = sum_j Tm[(i - j) mod grid][j] u[j]
    y_ref = np.zeros(32 * 32)
    for a, x in enumerate(idx):
        d = ((x[None, :] - idx) % np.array(shape))
        y_ref[a] = np.sum(Tm[d[:, 0] * 32 + d[:, 1], np.arange(32 * 32)] * u.reshape(-1))
    np.testing.assert_allclose(E.apply(u, w, h).reshape(-1), y_ref, atol=1e-12)
