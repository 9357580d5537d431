"""FP64 CPU oracle for the 2D complex DFT -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library's CUDA path shares no code
with it and never calls it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, built with
gcc into ``_build/liboracle.so``).  This module only marshals numpy arrays:
complex64 inputs are widened exactly to complex128 before every call.

Functions (all unnormalised, ``dir=-1`` forward, ``dir=+1`` inverse):

* :func:`fft1d_batch` -- recursive radix-2 Cooley-Tukey along the last axis.
* :func:`fft2d` -- rows then columns of each ``[ny][nx]`` slice (Section 5).
* :func:`dft1d_brute`, :func:`dft2d_brute` -- the O(N^2) definition.
* :func:`fft2d_rows`, :func:`fft2d_cols` -- selected output rows / columns of
  a 2D transform (definition along one axis, recursive FFT along the other).
* :func:`dft1d_bins` -- selected bins of one long 1D transform, each from the
  definition in one O(n) pass.
* :func:`fft1d_any`, :func:`fft2d_any` -- any length (not only powers of two):
  the recursion split by the smallest prime factor, primes from the definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "oracle.c")

_lib = None


def library_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (OpenMP on).  Returns the .so path."""
    out = library_path(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    d = ctypes.c_void_p
    L = ctypes.c_long
    i = ctypes.c_int
    lib.oracle_fft1d_batch.argtypes = [d, d, L, L, i, i]
    lib.oracle_fft2d.argtypes = [d, d, L, L, L, i, i]
    lib.oracle_dft1d_brute.argtypes = [d, d, L, i]
    lib.oracle_dft2d_brute.argtypes = [d, d, L, L, i]
    lib.oracle_fft2d_rows.argtypes = [d, d, L, L, d, L, i, i]
    lib.oracle_fft2d_cols.argtypes = [d, d, L, L, d, L, i, i]
    lib.oracle_dft1d_bins.argtypes = [d, d, L, d, L, i, i]
    lib.oracle_fft1d_any.argtypes = [d, d, L, L, i, i]
    lib.oracle_fft2d_any.argtypes = [d, d, L, L, L, i, i]
    for f in ("oracle_fft1d_batch", "oracle_fft2d", "oracle_dft1d_brute",
              "oracle_dft2d_brute", "oracle_fft2d_rows", "oracle_fft2d_cols",
              "oracle_dft1d_bins", "oracle_fft1d_any", "oracle_fft2d_any",
              "oracle_max_threads"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


def load(mutant: int = 0):
    """Load (building if needed) the oracle library; mutant != 0 loads a
    deliberately broken build used only to show that the pins catch it."""
    global _lib
    if mutant == 0 and _lib is not None:
        return _lib
    lib = _bind(ctypes.CDLL(build(mutant)))
    if mutant == 0:
        _lib = lib
    return lib


def max_threads() -> int:
    return int(load().oracle_max_threads())


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def fft1d_batch(x, dir: int = -1, threads: int = 1, lib=None) -> np.ndarray:
    """Transform along the last axis of ``x`` (any leading shape)."""
    lib = lib or load()
    a = _c128(x)
    n = a.shape[-1]
    out = np.empty_like(a)
    _check(lib.oracle_fft1d_batch(a.ctypes.data, out.ctypes.data, n, a.size // max(n, 1),
                                  dir, threads), "fft1d_batch")
    return out


def fft2d(x, dir: int = -1, threads: int = 1, lib=None) -> np.ndarray:
    """2D transform of each trailing ``[ny][nx]`` slice of ``x``."""
    lib = lib or load()
    a = _c128(x)
    ny, nx = a.shape[-2], a.shape[-1]
    batch = a.size // max(nx * ny, 1)
    out = np.empty_like(a)
    _check(lib.oracle_fft2d(a.ctypes.data, out.ctypes.data, nx, ny, batch, dir, threads),
           "fft2d")
    return out


def dft1d_brute(x, dir: int = -1, lib=None) -> np.ndarray:
    lib = lib or load()
    a = _c128(x).reshape(-1)
    out = np.empty_like(a)
    _check(lib.oracle_dft1d_brute(a.ctypes.data, out.ctypes.data, a.size, dir), "dft1d_brute")
    return out


def dft2d_brute(x, dir: int = -1, lib=None) -> np.ndarray:
    lib = lib or load()
    a = _c128(x)
    ny, nx = a.shape
    out = np.empty_like(a)
    _check(lib.oracle_dft2d_brute(a.ctypes.data, out.ctypes.data, nx, ny, dir), "dft2d_brute")
    return out


def fft2d_rows(x, ky, dir: int = -1, threads: int = 1, lib=None) -> np.ndarray:
    """Output rows ``X[ky, :]`` of the 2D transform of one ``[ny][nx]`` array."""
    lib = lib or load()
    a = _c128(x)
    ny, nx = a.shape
    k = np.ascontiguousarray(ky, dtype=np.int64).reshape(-1)
    out = np.empty((k.size, nx), dtype=np.complex128)
    _check(lib.oracle_fft2d_rows(a.ctypes.data, out.ctypes.data, nx, ny, k.ctypes.data,
                                 k.size, dir, threads), "fft2d_rows")
    return out


def fft2d_cols(x, kx, dir: int = -1, threads: int = 1, lib=None) -> np.ndarray:
    """Output columns ``X[:, kx]`` of the 2D transform, returned as ``[nk][ny]``."""
    lib = lib or load()
    a = _c128(x)
    ny, nx = a.shape
    k = np.ascontiguousarray(kx, dtype=np.int64).reshape(-1)
    out = np.empty((k.size, ny), dtype=np.complex128)
    _check(lib.oracle_fft2d_cols(a.ctypes.data, out.ctypes.data, nx, ny, k.ctypes.data,
                                 k.size, dir, threads), "fft2d_cols")
    return out


def dft1d_bins(x, bins, dir: int = -1, threads: int = 1, lib=None) -> np.ndarray:
    """Bins ``X[bins]`` of the 1D transform of the vector ``x`` (definition)."""
    lib = lib or load()
    a = _c128(x).reshape(-1)
    k = np.ascontiguousarray(bins, dtype=np.int64).reshape(-1)
    out = np.empty(k.size, dtype=np.complex128)
    _check(lib.oracle_dft1d_bins(a.ctypes.data, out.ctypes.data, a.size, k.ctypes.data, k.size,
                                 dir, threads), "dft1d_bins")
    return out


def fft1d_any(x, dir: int = -1, threads: int = 1, lib=None) -> np.ndarray:
    """Transform of any length along the last axis of ``x``."""
    lib = lib or load()
    a = _c128(x)
    n = a.shape[-1]
    out = np.empty_like(a)
    _check(lib.oracle_fft1d_any(a.ctypes.data, out.ctypes.data, n, a.size // max(n, 1), dir, threads),
           "fft1d_any")
    return out


def fft2d_any(x, dir: int = -1, threads: int = 1, lib=None) -> np.ndarray:
    """2D transform of each trailing ``[ny][nx]`` slice, any sizes."""
    lib = lib or load()
    a = _c128(x)
    ny, nx = a.shape[-2], a.shape[-1]
    out = np.empty_like(a)
    _check(lib.oracle_fft2d_any(a.ctypes.data, out.ctypes.data, nx, ny, a.size // max(nx * ny, 1), dir,
                                threads), "fft2d_any")
    return out
