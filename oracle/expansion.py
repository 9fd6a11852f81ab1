"""O1/O2/O3/O5/O6: the convolution-product expansion by definition (test infrastructure, FP64).

Readings (the paper leaves these implicit):
* Indices are 0-based and periodic: the discrete convolution of Section 3.5,
  v[i] = sum_j u[i-j] h[j], is read with j = 0..n-1 and i-j taken mod n
  (per axis in 2D).  h_k is given with its origin at index 0.
* The adjoint is not written in the paper, which only asks for products with
  H_m and H_m^* (Introduction; Corollaries 4.2/4.4).  For real h_k and w_k the
  adjoint of u -> h * (w . u) is v -> w . (h~ * v) with h~[i] = h[-i].
* The quadrature weight 1/P of the rectangle rule is folded into h_k by the
  input generators; O3 uses the same weight.

Every input is promoted to float64 before use.  Arrays are [B, *shape] for
right-hand sides and [m, *shape] for w and h; shape is (N,) or (Ny, Nx).
"""
from __future__ import annotations

import numpy as np

from . import dft as _dft


def _taps(hk: np.ndarray):
    """Offsets d (as index tuples) and values of the nonzero taps of h_k.

    Restricting the convolution sum to nonzero taps is exact: a zero tap adds
    exactly zero.
    """
    idx = np.nonzero(hk)
    return np.stack(idx, axis=-1), hk[idx]


def apply(u, w, h) -> np.ndarray:
    """O1: y = H_m u = sum_k h_k * (w_k . u)  (Eq. 1.4, discrete convolution of Section 3.5).

    y[b, i] = sum_k sum_j h_k[(i - j) mod n] w_k[j] u[b, j], evaluated as the
    shift sum y += h_k[d] * roll(w_k . u, d) over the taps d of h_k
    (roll(v, d)[i] = v[i - d], i.e. d = i - j).
    """
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    nd = w.ndim - 1
    axes = tuple(range(-nd, 0))
    y = np.zeros_like(u)
    for k in range(w.shape[0]):
        v = w[k] * u
        offs, vals = _taps(h[k])
        for d, hv in zip(offs, vals):
            y += hv * np.roll(v, tuple(int(t) for t in d), axis=axes)
    return y


def apply_adjoint(v, w, h) -> np.ndarray:
    """O2: x = H_m^* v = sum_k w_k . (h~_k * v), the transpose of O1.

    x[b, j] = sum_k w_k[j] sum_i h_k[(i - j) mod n] v[b, i]
            = sum_k w_k[j] sum_d h_k[d] v[b, j + d].
    """
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    nd = w.ndim - 1
    axes = tuple(range(-nd, 0))
    x = np.zeros_like(v)
    for k in range(w.shape[0]):
        t = np.zeros_like(v)
        offs, vals = _taps(h[k])
        for d, hv in zip(offs, vals):
            t += hv * np.roll(v, tuple(-int(s) for s in d), axis=axes)
        x += w[k] * t
    return x


def product_convolution(u, w, h) -> np.ndarray:
    """O6: the product-convolution form P_m u = sum_k w_k . (h_k * u) (Section 1,
    the kernel K(x, y) = sum_k w_k(x) h_k(x - y): windows on the output side).

    y[b, i] = sum_k w_k[i] sum_d h_k[d] u[b, i - d].
    """
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    nd = w.ndim - 1
    axes = tuple(range(-nd, 0))
    y = np.zeros_like(u)
    for k in range(w.shape[0]):
        t = np.zeros_like(u)
        offs, vals = _taps(h[k])
        for d, hv in zip(offs, vals):
            t += hv * np.roll(u, tuple(int(s) for s in d), axis=axes)
        y += w[k] * t
    return y


def product_convolution_adjoint(v, w, h) -> np.ndarray:
    """O6*: P_m^* v = sum_k h~_k * (w_k . v), the transpose of O6.

    x[b, j] = sum_k sum_d h_k[d] w_k[j + d] v[b, j + d].
    """
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    nd = w.ndim - 1
    axes = tuple(range(-nd, 0))
    x = np.zeros_like(v)
    for k in range(w.shape[0]):
        z = w[k] * v
        offs, vals = _taps(h[k])
        for d, hv in zip(offs, vals):
            x += hv * np.roll(z, tuple(-int(s) for s in d), axis=axes)
    return x


def _flat_index(idx: np.ndarray, shape) -> np.ndarray:
    return np.ravel_multi_index(tuple(np.moveaxis(idx, -1, 0)), shape)


def apply_at(u, w, h, points: np.ndarray) -> np.ndarray:
    """O1 at selected outputs only (gather form of the same sum).

    ``points`` is [S, ndims] integer output positions; returns [B, S]:
    y[b, i] = sum_k sum_d h_k[d] w_k[i - d] u[b, i - d].
    """
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    shape = w.shape[1:]
    nd = len(shape)
    pts = np.asarray(points).reshape(-1, nd)
    uf = u.reshape(u.shape[0], -1)
    out = np.zeros((u.shape[0], pts.shape[0]))
    for k in range(w.shape[0]):
        offs, vals = _taps(np.asarray(h[k]))
        src = (pts[:, None, :] - offs[None, :, :]) % np.asarray(shape)   # [S, T, nd]
        fi = _flat_index(src, shape)                                        # [S, T]
        wk = w[k].reshape(-1)[fi]                                           # [S, T]
        coef = wk * vals.astype(np.float64)[None, :]
        out += np.einsum("st,bst->bs", coef, uf[:, fi])
    return out


def apply_adjoint_at(v, w, h, points: np.ndarray) -> np.ndarray:
    """O2 at selected outputs only: x[b, j] = sum_k w_k[j] sum_d h_k[d] v[b, j + d]."""
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    shape = w.shape[1:]
    nd = len(shape)
    pts = np.asarray(points).reshape(-1, nd)
    vf = v.reshape(v.shape[0], -1)
    fp = _flat_index(pts, shape)
    out = np.zeros((v.shape[0], pts.shape[0]))
    for k in range(w.shape[0]):
        wk = w[k].reshape(-1)[fp]                                           # [S]
        if not np.any(wk):
            continue
        offs, vals = _taps(np.asarray(h[k]))
        dst = (pts[:, None, :] + offs[None, :, :]) % np.asarray(shape)
        fi = _flat_index(dst, shape)
        out += wk[None, :] * np.einsum("t,bst->bs", vals.astype(np.float64), vf[:, fi])
    return out


def quadrature(kernel, u, shape) -> np.ndarray:
    """O3: direct quadrature of Hu(x) = int K(x, y) u(y) dy (Eq. 1.1).

    (H u)[i] = sum_j K(x_i, y_j) u[j] * Delta on the periodic grid
    x_i = y_i = i/N (per axis), Delta = 1/P.  ``kernel(x, y)`` receives
    coordinate arrays of shape [P, ndims] (x) and [P, ndims] (y) broadcast
    as [P, 1, nd] and [1, P, nd], and returns the [P, P] matrix K(x_i, y_j).
    """
    u = np.asarray(u, dtype=np.float64)
    shape = tuple(shape)
    grids = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    pts = np.stack([g.reshape(-1) for g in grids], axis=-1)                # [P, nd]
    K = kernel(pts[:, None, :], pts[None, :, :])                           # [P, P]
    P = pts.shape[0]
    uf = u.reshape(-1, P)
    return (uf @ K.T / P).reshape(u.shape)


def apply_from_spectra(u, w, hhat, shape) -> np.ndarray:
    """O1 with the impulse responses given by their half spectra hhat_k = R2C(h_k).

    y = C2R( sum_k hhat_k . R2C(w_k . u) ), with the naive DFTs of O4 and the
    standard C2R (imaginary parts of the DC/Nyquist bins of the last axis
    discarded).  By the FFT convolution identity of Section 3.5 this equals
    O1 when hhat_k = R2C(h_k).  This is the parametrisation the gradient with
    respect to hhat_k refers to.
    """
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    nd = len(shape)
    acc = 0.0
    for k in range(w.shape[0]):
        acc = acc + np.asarray(hhat[k]) * _dft.rdft_nd(w[k] * u, nd)
    return _dft.irdft_nd(acc, tuple(shape))


def c2r_adjoint(r, shape) -> np.ndarray:
    """Gradient G = dL/dRe Z + i dL/dIm Z of L = <C2R(Z), r> for a real r.

    Last axis (from the C2R formula in oracle.dft.irdft): interior bins get
    (2/n) DFT(r)[c], the DC and Nyquist bins (1/n) Re DFT(r)[c].  Leading axes
    (inverse DFT, complex linear): multiply by the conjugate transpose of the
    inverse-DFT matrix, i.e. (1/n) times the forward DFT.
    """
    r = np.asarray(r, dtype=np.float64)
    nx = shape[-1]
    hx = nx // 2
    G = _dft.dft(r, axis=-1)[..., : hx + 1] / nx
    wgt = np.full(hx + 1, 2.0)
    wgt[0] = 1.0
    wgt[hx] = 1.0
    G = G * wgt
    G[..., 0] = G[..., 0].real
    G[..., hx] = G[..., hx].real
    for ax in range(-len(shape), -1):
        G = _dft.dft(G, axis=ax) / r.shape[ax]
    return G


def grad(u, w, h, r):
    """O5: gradients of L = sum_b <H_m u_b, r_b> (real inner product).

    Returns (du, dw, dh, dhhat):
    * du[b]     = H_m^* r_b                                   (O2)
    * dw_k[j]   = sum_b u_b[j] sum_i h_k[(i - j) mod n] r_b[i]
    * dh_k[d]   = sum_b sum_j w_k[j] u_b[j] r_b[j + d]
    * dhhat_k   = sum_b G_b . conj(R2C(w_k . u_b)), G_b = c2r_adjoint(r_b),
                  in the convention dL/dRe + i dL/dIm.
    """
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    shape = w.shape[1:]
    nd = len(shape)
    axes = tuple(range(-nd, 0))
    du = apply_adjoint(r, w, h)
    m = w.shape[0]
    dw = np.zeros_like(w)
    dh = np.zeros_like(h)
    G = c2r_adjoint(r, shape)
    dhhat = np.zeros((m,) + G.shape[1:], dtype=np.complex128)
    P = int(np.prod(shape))
    for k in range(m):
        offs, vals = _taps(h[k])
        t = np.zeros_like(r)
        for d, hv in zip(offs, vals):
            t += hv * np.roll(r, tuple(-int(s) for s in d), axis=axes)
        dw[k] = np.sum(u * t, axis=0)
        v = w[k] * u
        # dh_k[d] = sum_b sum_j v_b[j] r_b[j + d]: circular cross-correlation, by definition
        for flat in range(P):
            d = np.unravel_index(flat, shape)
            dh[k][d] = np.sum(v * np.roll(r, tuple(-int(s) for s in d), axis=axes))
        X = _dft.rdft_nd(v, nd)
        dhhat[k] = np.sum(G * np.conj(X), axis=0)
    return du, dw, dh, dhhat
