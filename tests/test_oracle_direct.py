"""Pins for the compiled FP64 oracle (oracle/direct.c): O1/O2 of Eq. 1.4.

The compiled oracle evaluates the same definitions as oracle/expansion.py.
It is pinned both against that oracle (two independent implementations of
the definition) and directly against what the paper and the mathematics fix:
the quadrature identity of Lemma 3.1, the Poisson-summation closed forms of a
pure convolution, the adjoint identity and the dense kernel matrix built
entry by entry.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import direct as C
from oracle import expansion as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rand(shape, m, batch, seed, sparse=True):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((m,) + shape)
    h = rng.standard_normal((m,) + shape)
    if sparse:
        h[rng.random(h.shape) < 0.6] = 0.0
        w[rng.random(w.shape) < 0.4] = 0.0
        w[0, : shape[0] // 3] = 0.0          # whole zero rows (or samples, 1D)
    u = rng.standard_normal((batch,) + shape)
    return w, h, u


def _relmax(a, b):
    """max |a - b| / max |b|; an all-zero reference must be matched exactly."""
    scale = np.max(np.abs(b))
    if scale == 0.0:
        return 0.0 if np.all(a == 0) else math.inf
    return float(np.max(np.abs(a - b)) / scale)


@pytest.mark.parametrize("shape", [(1,), (17,), (64,), (1, 9), (5, 7), (16, 24), (33, 20)])
def test_matches_numpy_oracle(shape):
    w, h, u = _rand(shape, 3, 2, 7 + len(shape))
    assert _relmax(C.apply(u, w, h), E.apply(u, w, h)) < 1e-13
    assert _relmax(C.apply_adjoint(u, w, h), E.apply_adjoint(u, w, h)) < 1e-13
    rng = np.random.default_rng(3)
    pts = np.stack([rng.integers(0, n, 25) for n in shape], axis=-1)
    assert _relmax(C.apply_at(u, w, h, pts), E.apply_at(u, w, h, pts)) < 1e-13
    assert _relmax(C.apply_adjoint_at(u, w, h, pts), E.apply_adjoint_at(u, w, h, pts)) < 1e-13


def test_dense_kernel_matrix_entry_by_entry():
    """Lemma 3.1 read on the grid: the response at i to a unit input at j is
    sum_k h_k[(i - j) mod n] w_k[j], and the adjoint is the transpose."""
    shape = (6, 8)
    m = 3
    w, h, _ = _rand(shape, m, 1, 21)
    P = int(np.prod(shape))
    eye = np.eye(P).reshape((P,) + shape)
    K = C.apply(eye, w, h).reshape(P, P).T            # column j = H e_j
    Ka = C.apply_adjoint(eye, w, h).reshape(P, P).T
    idx = np.indices(shape).reshape(2, -1).T
    ref = np.zeros((P, P))
    for a, x in enumerate(idx):
        for b, y in enumerate(idx):
            d = tuple((x - y) % np.array(shape))
            ref[a, b] = sum(h[k][d] * w[k][tuple(y)] for k in range(m))
    assert np.max(np.abs(K - ref)) < 1e-13
    assert np.max(np.abs(Ka - ref.T)) < 1e-13


def test_lemma_3_1_quadrature_of_rank_m_kernel():
    """Direct quadrature of K(x, y) = sum_k h_k(x - y) w_k(y) equals the expansion."""
    N, m = 64, 3
    sig = [0.03, 0.05, 0.02]
    shift = [0.0, 0.1, -0.15]

    def hfun(k, d):
        d = d - shift[k]
        d = d - np.floor(d + 0.5)
        return np.exp(-d ** 2 / (2 * sig[k] ** 2)) * (1 + 2 * d)

    def wfun(k, y):
        return np.sin(2 * np.pi * (k + 1) * y) + 0.3 * k

    grid = np.arange(N) / N
    h = np.stack([hfun(k, grid) / N for k in range(m)])
    w = np.stack([wfun(k, grid) for k in range(m)])
    u = np.random.default_rng(8).standard_normal((2, N))
    K = sum(hfun(k, grid[:, None] - grid[None, :]) * wfun(k, grid[None, :]) for k in range(m))
    y_quad = u @ K.T / N
    assert _relmax(C.apply(u, w, h), y_quad) < 1e-13


def test_pure_convolution_closed_forms():
    """m = 1, w = 1: Fourier modes are eigenvectors with the Poisson-summation symbols
    of the periodised Gaussian (1D) and of the rotated anisotropic PSF (2D)."""
    N, sigma = 128, 0.02
    h = synth.gaussian_psf_1d(N, sigma)[None]
    j = np.arange(N)
    for f0 in (0, 3, 17, 64):
        u = np.cos(2 * np.pi * f0 * j / N)[None]
        sym = sum(math.exp(-2 * math.pi ** 2 * sigma ** 2 * (f0 + l * N) ** 2) for l in range(-2, 3))
        assert np.max(np.abs(C.apply(u, np.ones((1, N)), h) - sym * u)) < 1e-13
        assert np.max(np.abs(C.apply_adjoint(u, np.ones((1, N)), h) - sym * u)) < 1e-13
    ny, nx = 32, 64
    sx, sy, th = 2.1, 1.5, 0.9
    h2 = synth.aniso_psf_2d(ny, nx, sx, sy, th)[None]
    c, s = math.cos(th), math.sin(th)
    S = np.array([[c * c * sx ** 2 + s * s * sy ** 2, c * s * (sx ** 2 - sy ** 2)],
                  [c * s * (sx ** 2 - sy ** 2), s * s * sx ** 2 + c * c * sy ** 2]])

    def sym2(fx, fy):
        tot = 0.0
        for lx in (-1, 0, 1):
            for ly in (-1, 0, 1):
                xi = np.array([fx / nx + lx, fy / ny + ly])
                tot += math.exp(-2 * math.pi ** 2 * xi @ S @ xi)
        return tot

    rows, cols = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for fx, fy in [(1, 0), (0, 1), (4, -3), (-7, 5)]:
        u = np.cos(2 * np.pi * (fx * cols / nx + fy * rows / ny))[None]
        y = C.apply(u, np.ones((1, ny, nx)), h2)
        assert np.max(np.abs(y - sym2(fx, fy) / sym2(0, 0) * u)) < 1e-12


def test_adjoint_identity_on_hat_windows():
    """<H u, v> = <u, H* v> for the 2D workload family (hats, anisotropic PSFs)."""
    pr = synth.problem_2d(64, 96, 16, 2, 31, "normal")
    v = np.random.default_rng(4).standard_normal(pr.u.shape)
    hu = C.apply(pr.u, pr.w, pr.h)
    hv = C.apply_adjoint(v, pr.w, pr.h)
    lhs = np.sum(hu * v)
    rhs = np.sum(pr.u.astype(np.float64) * hv)
    assert abs(lhs - rhs) < 1e-12 * np.sqrt(np.sum(hu ** 2) * np.sum(v ** 2))


def test_float32_inputs_are_promoted_exactly():
    w, h, u = _rand((12, 16), 2, 2, 41)
    w32, h32, u32 = (a.astype(np.float32) for a in (w, h, u))
    a = C.apply(u32, w32, h32)
    b = C.apply(u32.astype(np.float64), w32.astype(np.float64), h32.astype(np.float64))
    assert np.array_equal(a, b)


def test_result_does_not_depend_on_the_thread_count():
    """Each thread owns whole output rows and the sum order is fixed: one thread
    and all threads give the same bits."""
    code = ("import sys; sys.path.insert(0, %r); import numpy as np, synth; from oracle import direct as C;"
            "pr = synth.problem_2d(64, 64, 4, 1, 5, 'uniform');"
            "y = C.apply(pr.u, pr.w, pr.h); x = C.apply_adjoint(pr.u, pr.w, pr.h);"
            "sys.stdout.write((y.tobytes() + x.tobytes()).hex()[:: 7])" % ROOT)
    out = []
    for nt in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        out.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                  check=True).stdout)
    assert out[0] == out[1] and len(out[0]) > 1000
