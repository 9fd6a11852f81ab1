"""Pins for O4, the oracle's naive DFT (sign convention of the Fourier atoms, Section 2;
FFT convolution identity, Section 3.5)."""
import numpy as np
import pytest

from oracle import dft as D


@pytest.mark.parametrize("n", [1, 2, 8, 16, 30])
def test_delta_and_atoms(n):
    # DFT of a delta at 0 is all ones.
    x = np.zeros(n)
    x[0] = 1.0
    assert np.allclose(D.dft(x), np.ones(n), atol=1e-14)
    # x[j] = exp(+2 i pi f0 j / n) maps to n * delta[f - f0]: pins the minus sign of e_k.
    for f0 in range(n):
        x = np.exp(2j * np.pi * f0 * np.arange(n) / n)
        X = D.dft(x)
        ref = np.zeros(n, complex)
        ref[f0] = n
        assert np.max(np.abs(X - ref)) < 1e-12 * max(n, 1)


def test_matches_library_fft_and_roundtrip():
    rng = np.random.default_rng(0)
    for n in (4, 16, 64, 100):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        assert np.max(np.abs(D.dft(x) - np.fft.fft(x))) < 1e-12 * n
        assert np.max(np.abs(D.idft(D.dft(x)) - x)) < 1e-13
        # Parseval: sum |x|^2 = (1/n) sum |X|^2
        assert abs(np.sum(abs(x) ** 2) - np.sum(abs(D.dft(x)) ** 2) / n) < 1e-10


def test_real_transforms_match_library_convention():
    rng = np.random.default_rng(1)
    for shape in [(16,), (8, 16), (4, 32)]:
        x = rng.standard_normal(shape)
        assert np.allclose(D.rdft_nd(x, len(shape)), np.fft.rfftn(x), atol=1e-12)
        X = np.fft.rfftn(x)
        assert np.allclose(D.irdft_nd(X, shape), x, atol=1e-12)
        # Non-Hermitian half spectrum: the C2R definition discards the imaginary
        # parts of the DC and Nyquist bins of the last axis, as the library does.
        Z = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
        assert np.allclose(D.irdft_nd(Z, shape), np.fft.irfftn(Z, s=shape, axes=tuple(range(-len(shape), 0))), atol=1e-12)


def test_convolution_identity_by_brute_force():
    # Section 3.5: v = F_n((F_n^* h) . (F_n^* u)), v[i] = sum_j u[i-j] h[j] (periodic).
    rng = np.random.default_rng(2)
    n = 12
    h = rng.standard_normal(n)
    u = rng.standard_normal(n)
    v = [sum(u[(i - j) % n] * h[j] for j in range(n)) for i in range(n)]
    w = D.idft(D.dft(h) * D.dft(u))
    assert np.max(np.abs(w.real - np.array(v))) < 1e-13
    assert np.max(np.abs(w.imag)) < 1e-13


def test_dft_at_delta_atom_and_full_transform():
    """dft_at: a delta at j0 gives exp(-2 i pi j0 f / n); a pure atom gives n at its frequency."""
    n = 64
    x = np.zeros(n)
    x[5] = 1.0
    f = np.array([0, 1, 7, 32, 63])
    np.testing.assert_allclose(D.dft_at(x, f)[0:], np.exp(-2j * np.pi * 5 * f / n), atol=1e-13)
    atom = np.exp(2j * np.pi * 9 * np.arange(n) / n)
    got = D.dft_at(atom, [9, 10])
    np.testing.assert_allclose(got, [n, 0], atol=1e-11)
    rng = np.random.default_rng(4)
    y = rng.standard_normal((2, n))
    np.testing.assert_allclose(D.dft_at(y, range(n)), D.dft(y), atol=1e-11)
