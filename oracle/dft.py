"""O4: naive discrete Fourier transforms (test infrastructure, FP64).

Sign convention: the Fourier atom e_k(x) = exp(-2 i pi k x) (Section 2), so
the forward DFT is X[f] = sum_j x[j] exp(-2 i pi j f / n), unnormalised, and
the inverse carries the 1/n.  This is the reading under which the FFT
convolution identity of Section 3.5, v = F_n((F_n^* h) . (F_n^* u)), holds
(F_n^* the forward DFT, F_n the inverse).

Everything here is an O(n^2) matrix product with the DFT matrix built from
cos/sin of 2 pi (j f mod n) / n; the "mod n" keeps the angles small so that
the matrix entries are correctly rounded.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    """[n][n] complex128 matrix M[f, j] = exp(-+2 i pi (j f mod n) / n)."""
    j = np.arange(n)
    jf = np.outer(j, j) % n
    ang = 2.0 * np.pi * jf / n
    sgn = 1.0 if inverse else -1.0
    return np.cos(ang) + 1j * sgn * np.sin(ang)


def dft(x: np.ndarray, axis: int = -1) -> np.ndarray:
    """Forward DFT along ``axis``: X[f] = sum_j x[j] exp(-2 i pi j f / n)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[axis]
    M = dft_matrix(n)
    return np.moveaxis(np.tensordot(M, np.moveaxis(x, axis, 0), axes=(1, 0)), 0, axis)


def idft(X: np.ndarray, axis: int = -1) -> np.ndarray:
    """Inverse DFT along ``axis``: x[j] = (1/n) sum_f X[f] exp(+2 i pi j f / n)."""
    X = np.asarray(X, dtype=np.complex128)
    n = X.shape[axis]
    M = dft_matrix(n, inverse=True)
    return np.moveaxis(np.tensordot(M, np.moveaxis(X, axis, 0), axes=(1, 0)), 0, axis) / n


def rdft(x: np.ndarray) -> np.ndarray:
    """Real-input DFT of the last axis, half spectrum f = 0..n/2 (R2C)."""
    n = x.shape[-1]
    return dft(x, axis=-1)[..., : n // 2 + 1]


def dft_at(x: np.ndarray, freqs) -> np.ndarray:
    """Forward DFT of the last axis at selected frequencies only (same definition as ``dft``).

    X[..., s] = sum_j x[..., j] exp(-2 i pi (j f_s mod n) / n); one O(n) sum per
    frequency, for lengths whose full DFT matrix would not fit in memory.
    """
    x = np.asarray(x)
    n = x.shape[-1]
    j = np.arange(n, dtype=np.int64)
    out = np.empty(x.shape[:-1] + (len(freqs),), dtype=np.complex128)
    for s, f in enumerate(freqs):
        atom = np.exp(-2j * np.pi * ((j * int(f)) % n) / n)
        out[..., s] = x.astype(np.complex128) @ atom
    return out


def irdft(X: np.ndarray, n: int) -> np.ndarray:
    """Complex-to-real inverse of the last axis from the half spectrum (C2R).

    x[s] = (1/n) [ Re X[0] + Re X[n/2] (-1)^s + 2 sum_{c=1}^{n/2-1} Re(X[c] e^{2 i pi c s / n}) ].
    The imaginary parts of the DC and Nyquist bins are discarded; this is the
    standard C2R definition for a half spectrum.
    """
    X = np.asarray(X, dtype=np.complex128)
    h = n // 2
    s = np.arange(n)
    c = np.arange(1, h)
    ang = 2.0 * np.pi * (np.outer(c, s) % n) / n
    E = np.cos(ang) + 1j * np.sin(ang)                    # [h-1][n]
    out = X[..., 0:1].real + X[..., h:h + 1].real * ((-1.0) ** s)
    out = out + 2.0 * np.real(np.tensordot(X[..., 1:h], E, axes=(-1, 0)))
    return out / n


def dft_nd(x: np.ndarray, ndims: int) -> np.ndarray:
    """Forward DFT over the last ``ndims`` axes."""
    X = np.asarray(x, dtype=np.complex128)
    for ax in range(-ndims, 0):
        X = dft(X, axis=ax)
    return X


def idft_nd(X: np.ndarray, ndims: int) -> np.ndarray:
    """Inverse DFT over the last ``ndims`` axes."""
    x = np.asarray(X, dtype=np.complex128)
    for ax in range(-ndims, 0):
        x = idft(x, axis=ax)
    return x


def rdft_nd(x: np.ndarray, ndims: int) -> np.ndarray:
    """Real-input DFT over the last ``ndims`` axes, half spectrum along the last (x) axis."""
    X = rdft(np.asarray(x, dtype=np.float64))
    for ax in range(-ndims, -1):
        X = dft(X, axis=ax)
    return X


def irdft_nd(X: np.ndarray, shape: tuple) -> np.ndarray:
    """C2R over the last len(shape) axes: full inverse DFT on the leading axes, then irdft on x."""
    ndims = len(shape)
    A = np.asarray(X, dtype=np.complex128)
    for ax in range(-ndims, -1):
        A = idft(A, axis=ax)
    return irdft(A, shape[-1])
