"""Operator constructions and the paper's example kernels (test infrastructure, FP64).

* Examples 3.1-3.3 and the matrix behind Fig. 1 (the spectrum of J, the
  integral operator whose kernel is the TVIR T).
* Two constructions of T_m(x, y) = sum_k c_k(x) B_{1,m}(y - k/m) on the hat
  space B_{1,m} of Definition 2.2:
  - the L2 projection of T(x, .) (Corollary 4.3), also onto the B-spline
    spaces B_{alpha,m} of order alpha = 2, 3,
  - interpolation at the nodes y_k = k/m (Section 4, "Interpolation VS
    approximation"), for which c_k = T(., y_k) because the hats are
    cardinal (B_{1,m}(y_i - y_k) = delta_ik).

Readings of Fig. 1 (the figure's discretisation is not stated):
* n = 256 samples x_i = y_i = i/n - 1/2 on the identified interval [-1/2, 1/2).
* The matrix is T[i, j] = T(x_i, y_j) with every column scaled to unit sum.
* Example 3.1 uses exp(-x^2 / sigma(y)^2); with that profile the printed
  values are reproduced up to one global factor 2^(1/4).  (The text of
  Example 3.1 writes 2 sigma^2; that profile does not reproduce the data.)
* Example 3.2 is printed garbled; the data are reproduced by
  T = max(1 - 2|x|/sigma(y), 0) with sigma(y) = 0.1 + 0.3 (1 - 2|y|), factor 1.
* Example 3.3: indicator of the closed interval |y| <= 1/4, Gaussians
  exp(-x^2 / sigma_i^2); reproduced up to the same factor 2^(1/4).
"""
from __future__ import annotations

import numpy as np


FIG1_N = 256
FIG1_SCALE = {1: 2.0 ** 0.25, 2: 1.0, 3: 2.0 ** 0.25}


def example_tvir(example: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """T(x, y) of Examples 3.1-3.3 (up to a per-column constant), broadcast over x and y."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if example == 1:
        s = 0.08 + 0.02 * np.cos(2.0 * np.pi * y)
        return np.exp(-(x ** 2) / s ** 2)
    if example == 2:
        s = 0.1 + 0.3 * (1.0 - 2.0 * np.abs(y))
        return np.maximum(1.0 - 2.0 * np.abs(x) / s, 0.0)
    if example == 3:
        inside = np.abs(y) <= 0.25
        return np.where(inside, np.exp(-(x ** 2) / 0.05 ** 2), np.exp(-(x ** 2) / 0.1 ** 2))
    raise ValueError(example)


def fig1_matrix(example: int, n: int = FIG1_N) -> np.ndarray:
    """Column-normalised TVIR matrix T[i, j] = T(x_i, y_j) / sum_i T(x_i, y_j)."""
    t = np.arange(n, dtype=np.float64) / n - 0.5
    T = example_tvir(example, t[:, None], t[None, :])
    return T / T.sum(axis=0, keepdims=True)


def fig1_singular_values(example: int, n: int = FIG1_N) -> np.ndarray:
    """Singular values of the Fig. 1 matrix times the example's global factor."""
    s = np.linalg.svd(fig1_matrix(example, n), compute_uv=False)
    return s * FIG1_SCALE[example]


def hat_basis(n: int, m: int) -> np.ndarray:
    """[n][m] matrix of periodic hats B_{1,m}(y_j - k/m) on y_j = j/n."""
    y = np.arange(n, dtype=np.float64) / n
    t = y[:, None] - np.arange(m)[None, :] / m
    t = t - np.round(t)
    return np.maximum(0.0, 1.0 - m * np.abs(t))


def cardinal_bspline(alpha: int, u) -> np.ndarray:
    """B_{alpha,1}(u), the centred cardinal B-spline of order alpha on unit knot spacing
    (Definition 2.2 with m = 1: the (alpha + 1)-fold convolution of the indicator of
    [-1/2, 1/2]), written out as its textbook piecewise polynomial for alpha = 1, 2, 3.
    B_{alpha,m}(t) = B_{alpha,1}(m t)."""
    a = np.abs(np.asarray(u, dtype=np.float64))
    if alpha == 1:
        return np.maximum(0.0, 1.0 - a)
    if alpha == 2:
        return np.where(a <= 0.5, 0.75 - a ** 2, np.where(a <= 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    if alpha == 3:
        return np.where(a <= 1.0, 2.0 / 3.0 - a ** 2 + 0.5 * a ** 3,
                        np.where(a <= 2.0, (2.0 - a) ** 3 / 6.0, 0.0))
    raise ValueError("alpha must be 1, 2 or 3")


def bspline_basis(n: int, m: int, alpha: int = 1) -> np.ndarray:
    """[n][m] matrix of periodic B-splines B_{alpha,m}(y_j - k/m) on y_j = j/n
    (Definition 2.2, nodes k/m; m >= alpha + 2 keeps one bump per period)."""
    if m < alpha + 2:
        raise ValueError("Definition 2.2 needs m >= alpha + 2")
    y = np.arange(n, dtype=np.float64) / n
    t = y[:, None] - np.arange(m)[None, :] / m
    t = t - np.round(t)
    return cardinal_bspline(alpha, m * t)


def projection_coefficients(T: np.ndarray, m: int, alpha: int = 1) -> np.ndarray:
    """Coefficients of the L2 projection of every row T(x_i, .) onto the periodic
    B-splines of order alpha (Corollary 4.3; hats for alpha = 1):
    c(x_i) = argmin_c || T(x_i, .) - B c ||_2 on the sample grid,
    c = (B^T B)^{-1} B^T T(x_i, .).  Returns C [n][m] (h_k = C[:, k], w_k = B[:, k])."""
    B = hat_basis(T.shape[1], m) if alpha == 1 else bspline_basis(T.shape[1], m, alpha)
    return np.linalg.solve(B.T @ B, B.T @ np.asarray(T, dtype=np.float64).T).T


def project_on_hats(T: np.ndarray, m: int) -> np.ndarray:
    """L2 projection of every row T(x_i, .) onto span{B_{1,m}(. - k/m)} (Corollary 4.3):
    T_m = C B^T with C from projection_coefficients."""
    return projection_coefficients(T, m) @ hat_basis(T.shape[1], m).T


def project_on_bsplines(T: np.ndarray, m: int, alpha: int) -> np.ndarray:
    """L2 projection of every row T(x_i, .) onto span{B_{alpha,m}(. - k/m)} (Corollary 4.3)."""
    return projection_coefficients(T, m, alpha) @ bspline_basis(T.shape[1], m, alpha).T


def tensor_hat_basis(shape, gy: int, gx: int) -> np.ndarray:
    """[P][m] matrix of the 2D windows B_k(y) = B_{1,gy}(y1 - i/gy) B_{1,gx}(y2 - l/gx) on the
    grid y = (r/Ny, c/Nx), k = i gx + l (the tensor-product hats of Definition 2.2 per axis,
    flattened row-major over the grid)."""
    ny, nx = shape
    by = hat_basis(ny, gy)          # [ny][gy]
    bx = hat_basis(nx, gx)          # [nx][gx]
    return np.einsum("ri,cl->rcil", by, bx).reshape(ny * nx, gy * gx)


def projection_coefficients_2d(T: np.ndarray, shape, gy: int, gx: int) -> np.ndarray:
    """L2 projection of every row T(x_d, .) of a 2D TVIR onto the tensor-product hats
    (Corollary 4.3 with the 2D windows of tensor_hat_basis): c(d) = argmin_c ||T(d, .) - B c||
    on the sample grid, c = (B^T B)^{-1} B^T T(d, .).  T is [P][P] (shift d, input position
    j, both flattened row-major); returns C [P][m] (h_k = C[:, k] on the shift grid)."""
    B = tensor_hat_basis(shape, gy, gx)
    return np.linalg.solve(B.T @ B, B.T @ np.asarray(T, dtype=np.float64).T).T


def interpolate_on_hats(T: np.ndarray, m: int) -> np.ndarray:
    """Interpolation at the nodes y_k = k/m: T_m(x, y) = sum_k T(x, y_k) B_{1,m}(y - y_k).

    Requires the node positions to be samples (n divisible by m).
    """
    n = T.shape[1]
    if n % m:
        raise ValueError("nodes must be grid points")
    B = hat_basis(n, m)
    nodes = (np.arange(m) * n) // m
    return T[:, nodes] @ B.T


def svd_truncate(T: np.ndarray, m: int) -> np.ndarray:
    """Best rank-m approximation (Section 5.1: h_k = sigma_k f_k, w_k = e_k)."""
    U, s, Vt = np.linalg.svd(T)
    return (U[:, :m] * s[:m]) @ Vt[:m]


def svd_terms(T: np.ndarray, m: int, rank_tol: float = 1e-12):
    """The m leading terms of the SVD of T (Section 5.1), as an expansion:
    h [m][n] with h_k = sigma_k f_k (f_k the left singular vectors, over the
    shift d), w [m][n] with w_k = e_k (right singular vectors, over the input
    position j), and sigma [m], so that T[d][j] ~ sum_k h_k[d] w_k[j].  Each
    pair's sign is fixed by sum_j w_k[j] >= 0; terms with sigma_k <=
    rank_tol * sigma_1 (beyond the numerical rank) are zero."""
    U, s, Vt = np.linalg.svd(np.asarray(T, dtype=np.float64))
    n = T.shape[1]
    h = np.zeros((m, T.shape[0]))
    w = np.zeros((m, n))
    sig = np.zeros(m)
    for k in range(min(m, s.size)):
        if not s[k] > rank_tol * s[0]:
            continue
        sgn = -1.0 if Vt[k].sum() < 0 else 1.0
        sig[k] = s[k]
        h[k] = sgn * s[k] * U[:, k]
        w[k] = sgn * Vt[k]
    return h, w, sig
