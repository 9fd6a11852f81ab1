"""O1/O2 by direct FP64 summation in compiled C with OpenMP (test infrastructure).

The same plain definitions as ``oracle.expansion.apply`` / ``apply_adjoint``
/ ``apply_at`` / ``apply_adjoint_at`` (Eq. 1.4 with the discrete convolution
of Section 3.5, 0-based and periodic; the adjoint is its transpose), written
in C (``direct.c``) so that full-size grids finish in seconds on a many-core
host.  Pinned by ``tests/test_oracle_direct.py``: against the numpy oracle on
small grids, and directly against the Lemma 3.1 quadrature identity, the
Poisson-summation closed form, the adjoint identity and brute force.

Only the test suite, the smoke check and the CPU legs of the benchmark use
this module.  ``build()`` compiles ``direct.c`` with the host C compiler
(OpenMP when available) into ``oracle/_lib``; the thread count is OpenMP's
default (all cores of the process's affinity mask) unless ``OMP_NUM_THREADS``
says otherwise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "direct.c")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liboracle_direct.so")
_lib = None
_openmp = None


def build(force: bool = False) -> str:
    """Compile direct.c (gcc -O2, OpenMP if the compiler has it); returns the library path."""
    global _openmp
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + f".{os.getpid()}.tmp"
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", SRC, "-o", tmp]
    res = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    _openmp = res.returncode == 0
    if not _openmp:
        res = subprocess.run(base, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("oracle C build failed:\n" + res.stderr)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i = ctypes.c_int
        lib.pce_oracle_apply.argtypes = [i, i, i, i, i, P, i, P, i, P, i, P]
        lib.pce_oracle_apply.restype = i
        lib.pce_oracle_apply_at.argtypes = [i, i, i, i, i, P, i, P, i, P, i, P, ctypes.c_int64, P]
        lib.pce_oracle_apply_at.restype = i
        lib.pce_oracle_threads.argtypes = []
        lib.pce_oracle_threads.restype = i
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the parallel loops use."""
    return int(_load().pce_oracle_threads())


def _arr(a):
    """(contiguous float32 or float64 array, is-float64 flag)."""
    a = np.asarray(a)
    if a.dtype == np.float32:
        return np.ascontiguousarray(a), 0
    return np.ascontiguousarray(a, dtype=np.float64), 1


def _grid(w):
    w = np.asarray(w)
    shape = w.shape[1:]
    if len(shape) == 1:
        return 1, shape[0]
    if len(shape) == 2:
        return shape
    raise ValueError("w must be [m][N] or [m][Ny][Nx]")


def _run(adjoint: bool, u, w, h) -> np.ndarray:
    ny, nx = _grid(w)
    ua, u64 = _arr(u)
    wa, w64 = _arr(w)
    ha, h64 = _arr(h)
    m = wa.shape[0]
    if ha.shape != wa.shape or ua.shape[1:] != wa.shape[1:]:
        raise ValueError("shapes of u, w and h do not match")
    out = np.empty(ua.shape, dtype=np.float64)
    st = _load().pce_oracle_apply(int(adjoint), ua.shape[0], ny, nx, m, ua.ctypes.data, u64, wa.ctypes.data, w64,
                                  ha.ctypes.data, h64, out.ctypes.data)
    if st != 0:
        raise MemoryError("oracle: out of host memory")
    return out


def apply(u, w, h) -> np.ndarray:
    """O1: y = H_m u = sum_k h_k * (w_k . u)  (Eq. 1.4), all outputs, [B, *shape] float64."""
    return _run(False, u, w, h)


def apply_adjoint(v, w, h) -> np.ndarray:
    """O2: x = H_m^* v = sum_k w_k . (h~_k * v), all outputs, [B, *shape] float64."""
    return _run(True, v, w, h)


def _run_at(adjoint: bool, u, w, h, points) -> np.ndarray:
    ny, nx = _grid(w)
    ua, u64 = _arr(u)
    wa, w64 = _arr(w)
    ha, h64 = _arr(h)
    pts = np.asarray(points, dtype=np.int64).reshape(-1, 2 if ny > 1 or np.asarray(w).ndim == 3 else 1)
    if pts.shape[1] == 1:
        pts = np.concatenate([np.zeros_like(pts), pts], axis=1)
    pts = np.ascontiguousarray(pts)
    if np.any(pts[:, 0] < 0) or np.any(pts[:, 0] >= ny) or np.any(pts[:, 1] < 0) or np.any(pts[:, 1] >= nx):
        raise ValueError("points outside the grid")
    out = np.empty((ua.shape[0], pts.shape[0]), dtype=np.float64)
    st = _load().pce_oracle_apply_at(int(adjoint), ua.shape[0], ny, nx, wa.shape[0], ua.ctypes.data, u64,
                                     wa.ctypes.data, w64, ha.ctypes.data, h64, pts.ctypes.data, pts.shape[0],
                                     out.ctypes.data)
    if st != 0:
        raise MemoryError("oracle: out of host memory")
    return out


def apply_at(u, w, h, points) -> np.ndarray:
    """O1 at selected outputs ([S, ndims] integer positions): [B, S] float64."""
    return _run_at(False, u, w, h, points)


def apply_adjoint_at(v, w, h, points) -> np.ndarray:
    """O2 at selected outputs ([S, ndims] integer positions): [B, S] float64."""
    return _run_at(True, v, w, h, points)
