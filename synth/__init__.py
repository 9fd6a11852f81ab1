"""Seeded synthetic inputs for the convolution-product expansion.

This module builds the *inputs* of the operator H_m u = sum_k h_k * (w_k . u)
(Eq. 1.4): the windows w_k, the impulse responses h_k and the right-hand sides
u.  It holds none of the apply arithmetic (no convolution, no FFT).  Both the
FP64 oracle and the CUDA path consume exactly the arrays returned here.

Conventions
-----------
* Grids are periodic.  1D arrays are ``[N]``; 2D arrays are ``[Ny][Nx]``
  (row-major, x fastest).  A point (row, col) sits at y = (y1, y2) =
  (col/Nx, row/Ny) in [0,1)^2.
* Every array is generated in float64 and rounded to float32 once.
* ``h_k`` is stored with its origin at index 0 and negative offsets wrapped
  (offset -d lives at index N-d).
* Windows are periodic hats B_{1,m}(t - k/m), the order-1 cardinal B-spline
  of Definition 2.2 (peak 1, support 2/m, partition of unity).  In 2D the
  windows are tensor products on a gy x gx node grid, k = a*gx + c for the
  node at (row a/gy, col c/gx).
* h_k is the impulse response at the node: h_k = T(., y_k), the interpolation
  construction of Section 4 ("Interpolation VS approximation") combined with
  Lemma 3.1 (T_m(x, y) = sum_k h_k(x) w_k(y)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1604_04374


def rng_for(index: int) -> np.random.Generator:
    """PCG64 generator seeded with SEED_BASE + index."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(index)))


# ----------------------------------------------------------------- windows

def hat_1d(n: int, m: int, k: int) -> np.ndarray:
    """Periodic hat B_{1,m}(x - k/m) sampled at x_i = i/n (float64).

    B_{1,m}(t) = max(0, 1 - m|t|) for the periodic distance |t| in [0, 1/2]
    (Definition 2.2 with alpha = 1: m * B_{0,m} * B_{0,m}, B_{0,m} the
    indicator of [-1/(2m), 1/(2m)]).
    """
    x = np.arange(n, dtype=np.float64) / n
    t = x - k / m
    t = t - np.round(t)          # periodic distance, t in [-1/2, 1/2]
    return np.maximum(0.0, 1.0 - m * np.abs(t))


def hat_windows_1d(n: int, m: int) -> np.ndarray:
    """[m][n] float32 hats centred at y_k = k/m, k = 0..m-1."""
    return np.stack([hat_1d(n, m, k) for k in range(m)]).astype(np.float32)


def node_grid(m: int) -> tuple[int, int]:
    """Node grid (gy, gx) for m 2D windows: gy = 2^ceil(log2(m)/2), gx = m/gy."""
    if m < 1 or (m & (m - 1)) != 0:
        raise ValueError("m must be a power of two for a 2D node grid")
    gy = 1 << math.ceil(math.log2(m) / 2)
    return gy, m // gy


def hat_windows_2d(ny: int, nx: int, gy: int, gx: int) -> np.ndarray:
    """[gy*gx][ny][nx] float32 tensor-product hats B_{1,gy}(row) B_{1,gx}(col)."""
    out = np.empty((gy * gx, ny, nx), dtype=np.float64)
    for a in range(gy):
        wr = hat_1d(ny, gy, a)
        for c in range(gx):
            wc = hat_1d(nx, gx, c)
            out[a * gx + c] = np.outer(wr, wc)
    return out.astype(np.float32)


def hat_factors_2d(ny: int, nx: int, gy: int, gx: int) -> tuple[np.ndarray, np.ndarray]:
    """Factors of the tensor-product hats: wy [m][ny], wx [m][nx] float32 with
    hat_windows_2d(...)[k] == outer(wy[k], wx[k]) exactly (the hat values are
    dyadic rationals, so the products are exact in float32)."""
    m = gy * gx
    wy = np.empty((m, ny), dtype=np.float32)
    wx = np.empty((m, nx), dtype=np.float32)
    for a in range(gy):
        for c in range(gx):
            wy[a * gx + c] = hat_1d(ny, gy, a)
            wx[a * gx + c] = hat_1d(nx, gx, c)
    return wy, wx


# ------------------------------------------------------ impulse responses

def sigma_1d(y: float) -> float:
    """sigma(y) = 0.01 + 0.005 sin(2 pi y): the 1D space-varying blur width."""
    return 0.01 + 0.005 * math.sin(2.0 * math.pi * y)


def gaussian_psf_1d(n: int, sigma: float) -> np.ndarray:
    """Periodised unit-mass Gaussian impulse response, times the quadrature weight 1/n.

    h[i] = g_sigma(d_i) / n with d_i = i/n wrapped to [-1/2, 1/2) and
    g_sigma(d) = sum_{j in {-1,0,1}} (2 pi sigma^2)^(-1/2) exp(-(d+j)^2 / (2 sigma^2)).
    """
    x = np.arange(n, dtype=np.float64) / n
    d = x - np.floor(x + 0.5)
    g = np.zeros(n, dtype=np.float64)
    for j in (-1.0, 0.0, 1.0):
        g += np.exp(-((d + j) ** 2) / (2.0 * sigma * sigma))
    g /= math.sqrt(2.0 * math.pi) * sigma
    return g / n


def psf_params_2d(y1: float, y2: float) -> tuple[float, float, float]:
    """(sigma_x, sigma_y, theta) of the anisotropic PSF at y = (y1, y2), in pixels."""
    return 1.5 + 1.0 * y1, 1.5 + 1.0 * y2, math.pi * y1 * y2


def aniso_psf_2d(ny: int, nx: int, sx: float, sy: float, theta: float) -> np.ndarray:
    """Rotated anisotropic Gaussian PSF with unit discrete sum, origin at [0,0].

    Covariance S = R(theta) diag(sx^2, sy^2) R(theta)^T in the (col, row)
    pixel axes, R the counter-clockwise rotation.  Evaluated at the
    minimum-image offsets (dx, dy) in [-nx/2, nx/2) x [-ny/2, ny/2).
    """
    dx = np.arange(nx, dtype=np.float64)
    dx = dx - nx * (dx >= nx // 2)
    dy = np.arange(ny, dtype=np.float64)
    dy = dy - ny * (dy >= ny // 2)
    c, s = math.cos(theta), math.sin(theta)
    # inverse covariance R diag(1/sx^2, 1/sy^2) R^T
    a11 = c * c / sx**2 + s * s / sy**2
    a22 = s * s / sx**2 + c * c / sy**2
    a12 = c * s * (1.0 / sx**2 - 1.0 / sy**2)
    X = dx[None, :]
    Y = dy[:, None]
    q = a11 * X * X + 2.0 * a12 * X * Y + a22 * Y * Y
    g = np.exp(-0.5 * q)
    return g / g.sum()


# --------------------------------------------------------------- problems

@dataclass
class Problem:
    """One synthetic convolution-product problem (float32 arrays)."""
    name: str
    shape: tuple            # (N,) or (Ny, Nx)
    m: int
    w: np.ndarray           # [m, *shape]
    h: np.ndarray           # [m, *shape]
    u: np.ndarray           # [B, *shape]
    meta: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return int(self.u.shape[0])


def problem_1d(n: int, m: int, batch: int, seed_index: int, dist: str = "normal") -> Problem:
    """1D problem: m hats at k/m, h_k = periodised Gaussian with sigma(y_k)."""
    w = hat_windows_1d(n, m)
    h = np.stack([gaussian_psf_1d(n, sigma_1d(k / m)) for k in range(m)]).astype(np.float32)
    u = draw(rng_for(seed_index), (batch, n), dist)
    return Problem(f"1d_n{n}_m{m}_b{batch}", (n,), m, w, h, u, {"dist": dist})


def problem_2d(ny: int, nx: int, m: int, batch: int, seed_index: int,
               dist: str = "uniform", grid: tuple[int, int] | None = None) -> Problem:
    """2D problem: m tensor hats on a node grid, h_k = anisotropic PSF at node k."""
    gy, gx = grid if grid is not None else node_grid(m)
    if gy * gx != m:
        raise ValueError("node grid does not hold m windows")
    w = hat_windows_2d(ny, nx, gy, gx)
    h = np.empty((m, ny, nx), dtype=np.float32)
    for a in range(gy):
        for c in range(gx):
            sx, sy, th = psf_params_2d(c / gx, a / gy)
            h[a * gx + c] = aniso_psf_2d(ny, nx, sx, sy, th).astype(np.float32)
    u = draw(rng_for(seed_index), (batch, ny, nx), dist)
    return Problem(f"2d_{ny}x{nx}_m{m}_b{batch}", (ny, nx), m, w, h, u,
                   {"dist": dist, "grid": (gy, gx)})


def draw(rng: np.random.Generator, shape, dist: str) -> np.ndarray:
    """u ~ N(0,1) ('normal') or U[0,1) ('uniform'), drawn in float64, rounded to float32."""
    if dist == "normal":
        x = rng.standard_normal(shape)
    elif dist == "uniform":
        x = rng.random(shape)
    else:
        raise ValueError(dist)
    return x.astype(np.float32)


# Named workloads (seed index = position in the list of workloads).
WORKLOADS = {
    # 1D N=1024, m=8 hats, periodised Gaussian sigma(y)=0.01+0.005 sin(2 pi y), B=1, u~N(0,1)
    "1d_n1024_m8_b1": lambda: problem_1d(1024, 8, 1, 0, "normal"),
    # 2D 1024x1024, B=8, m=16 hats on 4x4 nodes, anisotropic PSF, u~U[0,1)
    "2d_1024_m16_b8": lambda: problem_2d(1024, 1024, 16, 8, 1, "uniform", (4, 4)),
    # 2D 512x512, B=16, m=16 hats on 4x4 nodes, same PSF family
    "2d_512_m16_b16": lambda: problem_2d(512, 512, 16, 16, 2, "uniform", (4, 4)),
    # 2D 2048x2048, B=4, m=64 hats on 8x8 nodes, u~N(0,1)
    "2d_2048_m64_b4": lambda: problem_2d(2048, 2048, 64, 4, 3, "normal", (8, 8)),
}


def workload(name: str) -> Problem:
    return WORKLOADS[name]()


# ------------------------------------------------------------ uneven batches

BATCH_SHAPES = ((4096,), (16384,), (65536,), (256, 256), (512, 512), (1024, 1024))
BATCH_M = (4, 8, 16, 32)


@dataclass
class BatchMix:
    """Uneven tasks: task i applies operator ops[op_of[i]] (forward or adjoint) to inputs[i] (B = 1)."""
    name: str
    ops: list            # [(shape, m, w [m,*shape] f32, h [m,*shape] f32)]
    op_of: list          # [n_tasks] operator index
    adjoint: list        # [n_tasks] bool
    inputs: list         # [n_tasks] arrays [1, *shape] f32


def batch_operator(shape: tuple, m: int):
    """(w, h) of one operator of the mix: 1D hats + periodised Gaussians as in the
    1D workload, 2D tensor hats on node_grid(m) + the anisotropic PSF family."""
    if len(shape) == 1:
        pr = problem_1d(shape[0], m, 1, 0)
        return pr.w, pr.h
    gy, gx = node_grid(m)
    w = hat_windows_2d(shape[0], shape[1], gy, gx)
    h = np.empty((m,) + tuple(shape), dtype=np.float32)
    for a in range(gy):
        for c in range(gx):
            sx, sy, th = psf_params_2d(c / gx, a / gy)
            h[a * gx + c] = aniso_psf_2d(shape[0], shape[1], sx, sy, th).astype(np.float32)
    return w, h


def batch_mix(n_tasks: int = 256, seed_index: int = 4, shapes=BATCH_SHAPES, ms=BATCH_M) -> BatchMix:
    """n_tasks tasks with shape, m and direction drawn uniformly from a seed;
    inputs u ~ N(0,1) in 1D and U[0,1) in 2D, one right-hand side each."""
    rng = rng_for(seed_index)
    picks = [(int(rng.integers(len(shapes))), int(rng.integers(len(ms))), bool(rng.integers(2)))
             for _ in range(n_tasks)]
    keys = sorted({(s, k) for s, k, _ in picks})
    index = {key: i for i, key in enumerate(keys)}
    ops = []
    for s, k in keys:
        w, h = batch_operator(shapes[s], ms[k])
        ops.append((tuple(shapes[s]), ms[k], w, h))
    op_of = [index[(s, k)] for s, k, _ in picks]
    adjoint = [a for _, _, a in picks]
    inputs = [draw(rng, (1,) + tuple(shapes[s]), "normal" if len(shapes[s]) == 1 else "uniform")
              for s, _, _ in picks]
    return BatchMix(f"batch{n_tasks}_mixed", ops, op_of, adjoint, inputs)


# ----------------------------------------------- wavelet windows (Section 4.3)

# Daubechies' orthonormal scaling filter with two vanishing moments (D4), closed form.
_S3 = math.sqrt(3.0)
D4_FILTER = np.array([1 + _S3, 3 + _S3, 3 - _S3, 1 - _S3]) / (4 * math.sqrt(2.0))


def _synthesis_step(a: np.ndarray, d: np.ndarray, hfil: np.ndarray) -> np.ndarray:
    """One periodic inverse DWT step: length L coefficients -> length 2L signal,
    x[t] = sum_k a[k] h[t - 2k] + d[k] g[t - 2k] (indices mod 2L), g[i] = (-1)^i h[M-1-i]."""
    L = a.shape[0]
    M = hfil.shape[0]
    g = np.array([(-1) ** i * hfil[M - 1 - i] for i in range(M)])
    x = np.zeros(2 * L)
    for k in range(L):
        for i in range(M):
            t = (2 * k + i) % (2 * L)
            x[t] += a[k] * hfil[i] + d[k] * g[i]
    return x


def periodic_wavelet(n: int, j: int, k: int, kind: str, hfil: np.ndarray = D4_FILTER) -> np.ndarray:
    """Periodic orthonormal scaling function ('phi') or wavelet ('psi') at scale j,
    position k < 2^j, sampled on n = 2^L points (float64): the inverse periodic DWT
    of a unit coefficient, synthesised up to length n."""
    L = int(round(math.log2(n)))
    if 2 ** L != n or not 0 <= j < L or not 0 <= k < 2 ** j:
        raise ValueError("need n = 2^L, 0 <= j < L, 0 <= k < 2^j")
    a = np.zeros(2 ** j)
    d = np.zeros(2 ** j)
    (a if kind == "phi" else d)[k] = 1.0
    x = _synthesis_step(a, d, hfil)
    while x.shape[0] < n:
        x = _synthesis_step(x, np.zeros_like(x), hfil)
    return x


def wavelet_windows_1d(n: int, j0: int, levels: int) -> tuple[np.ndarray, list]:
    """Windows of the wavelet form (Section 4.3): the 2^j0 scaling functions at scale j0
    and the wavelets of scales j0 .. j0+levels-1 (2^j each), periodic D4.
    Returns ([m][n] float32, [(kind, j, k)])."""
    funcs, labels = [], []
    for k in range(2 ** j0):
        funcs.append(periodic_wavelet(n, j0, k, "phi"))
        labels.append(("phi", j0, k))
    for j in range(j0, j0 + levels):
        for k in range(2 ** j):
            funcs.append(periodic_wavelet(n, j, k, "psi"))
            labels.append(("psi", j, k))
    return np.stack(funcs).astype(np.float32), labels


def wavelet_windows_2d(ny: int, nx: int, j0: int, levels: int) -> tuple[np.ndarray, list]:
    """Tensor-product windows phi_{j0,a}(row) phi_{j0,c}(col) and psi_{j,a}(row) psi_{j,c}(col),
    j = j0 .. j0+levels-1: supports from most of the grid down to 3/2^j of each side."""
    funcs, labels = [], []
    for a in range(2 ** j0):
        fa = periodic_wavelet(ny, j0, a, "phi")
        for c in range(2 ** j0):
            funcs.append(np.outer(fa, periodic_wavelet(nx, j0, c, "phi")))
            labels.append(("phi", j0, a, c))
    for j in range(j0, j0 + levels):
        for a in range(2 ** j):
            fa = periodic_wavelet(ny, j, a, "psi")
            for c in range(2 ** j):
                funcs.append(np.outer(fa, periodic_wavelet(nx, j, c, "psi")))
                labels.append(("psi", j, a, c))
    return np.stack(funcs).astype(np.float32), labels


def wavelet_problem(shape: tuple, j0: int, levels: int, batch: int, seed_index: int,
                    radius: int | None = None) -> Problem:
    """Wavelet windows of varying support with random impulse responses supported on
    |offset| <= radius per axis (default 12 in 1D, 5 in 2D); u ~ N(0,1)."""
    if radius is None:
        radius = 12 if len(shape) == 1 else 5
    if len(shape) == 1:
        w, labels = wavelet_windows_1d(shape[0], j0, levels)
    else:
        w, labels = wavelet_windows_2d(shape[0], shape[1], j0, levels)
    m = w.shape[0]
    rng = rng_for(seed_index)
    h = np.zeros((m,) + tuple(shape), np.float32)
    offs = [np.arange(-radius, radius + 1) % n for n in shape]
    if len(shape) == 1:
        h[:, offs[0]] = rng.standard_normal((m, offs[0].size)).astype(np.float32)
    else:
        h[:, offs[0][:, None], offs[1][None, :]] = rng.standard_normal(
            (m, offs[0].size, offs[1].size)).astype(np.float32)
    u = draw(rng, (batch,) + tuple(shape), "normal")
    return Problem(f"wavelet_{'x'.join(map(str, shape))}_j{j0}_l{levels}", tuple(shape), m, w, h, u,
                   {"labels": labels})
