"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the transform itself: it only draws the
inputs (the paper names no dataset, so the workloads are synthetic), and both
the CUDA path and the FP64 oracle receive the same arrays from here.

Every generator takes an explicit integer seed and uses numpy's PCG64 bit
generator.  Uniform values are drawn directly as float32 in ``[0, 1)`` (a
multiple of 2**-24), so ``2u - 1`` in ``[-1, 1)`` is exact in float32.  Complex
arrays are complex64 with independent real and imaginary parts.

Recipes (sizes and distributions of the workloads; default seed 2506):

* ``uniform_complex`` -- re/im i.i.d. U[-1, 1).
* ``normal_complex``  -- re/im i.i.d. N(0, 1).
* ``exp_mix_2d`` / ``exp_mix_1d`` -- U[-1, 1) noise plus 8 unit-amplitude
  complex exponentials at distinct random integer frequencies (per array in
  2D, per signal for a batch of 1D signals), summed in float64 and rounded
  once to complex64.
* ``mask`` -- float32 U[0, 1) weights.
* ``ragged_exponents`` -- (log2 nx, log2 ny) pairs, each exponent i.i.d.
  uniform on {lo, ..., hi}.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 2506


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_complex(shape, seed: int = DEFAULT_SEED) -> np.ndarray:
    rng = _rng(seed)
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    out = np.empty(shape, dtype=np.complex64)
    v = out.view(np.float32).reshape(-1)
    # draw in chunks to keep the float32 scratch small for GB-sized arrays
    step = 1 << 24
    for s in range(0, v.size, step):
        u = rng.random(min(step, v.size - s), dtype=np.float32)
        v[s:s + u.size] = 2.0 * u - 1.0
    return out


def normal_complex(shape, seed: int = DEFAULT_SEED) -> np.ndarray:
    rng = _rng(seed)
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    out = np.empty(shape, dtype=np.complex64)
    v = out.view(np.float32).reshape(-1)
    step = 1 << 24
    for s in range(0, v.size, step):
        v[s:s + min(step, v.size - s)] = rng.standard_normal(min(step, v.size - s),
                                                             dtype=np.float32)
    return out


def mask(shape, seed: int = DEFAULT_SEED) -> np.ndarray:
    rng = _rng(seed)
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    return rng.random(shape, dtype=np.float32)


def _distinct_ints(rng: np.random.Generator, rows: int, k: int, n: int) -> np.ndarray:
    """rows x k integers in [0, n), distinct within each row (k <= n)."""
    f = rng.integers(0, n, size=(rows, k), dtype=np.int64)
    while True:
        s = np.sort(f, axis=1)
        bad = np.any(s[:, 1:] == s[:, :-1], axis=1) if k > 1 else np.zeros(rows, bool)
        if not bad.any():
            return f
        f[bad] = rng.integers(0, n, size=(int(bad.sum()), k), dtype=np.int64)


def _unit_roots(n: int) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    return np.exp(2j * np.pi * k / n)


def exp_mix_2d(ny: int, nx: int, seed: int = DEFAULT_SEED, n_exp: int = 8):
    """U[-1,1) noise + ``n_exp`` unit exponentials exp(+2*pi*i*(fx*x/nx + fy*y/ny)).

    Returns ``(x, freqs)`` with ``freqs`` an ``[n_exp, 2]`` array of (fy, fx).
    Under the forward (sign -1) transform each exponential contributes exactly
    ``nx*ny`` at bin (fy, fx).
    """
    rng = _rng(seed)
    noise = uniform_complex((ny, nx), seed=int(rng.integers(0, 2**62)))
    flat = _distinct_ints(rng, 1, min(n_exp, nx * ny), nx * ny)[0]
    freqs = np.stack([flat // nx, flat % nx], axis=1)
    tx, ty = _unit_roots(nx), _unit_roots(ny)
    xs = np.arange(nx, dtype=np.int64)
    out = np.empty((ny, nx), dtype=np.complex64)
    blk = max(1, (1 << 22) // nx)
    for y0 in range(0, ny, blk):
        ys = np.arange(y0, min(ny, y0 + blk), dtype=np.int64)
        acc = noise[y0:y0 + ys.size].astype(np.complex128)
        for fy, fx in freqs:
            acc += ty[(fy * ys) % ny][:, None] * tx[(fx * xs) % nx][None, :]
        out[y0:y0 + ys.size] = acc
    return out, freqs


def exp_mix_1d(batch: int, n: int, seed: int = DEFAULT_SEED, n_exp: int = 8):
    """``batch`` signals of length ``n``: U[-1,1) noise + ``n_exp`` unit
    exponentials exp(+2*pi*i*f*j/n) per signal, frequencies drawn per signal.

    Returns ``(x, freqs)`` with ``freqs`` of shape ``[batch, n_exp]``.
    """
    rng = _rng(seed)
    noise = uniform_complex((batch, n), seed=int(rng.integers(0, 2**62)))
    freqs = _distinct_ints(rng, batch, min(n_exp, n), n)
    t = _unit_roots(n)
    j = np.arange(n, dtype=np.int64)
    out = np.empty((batch, n), dtype=np.complex64)
    blk = max(1, (1 << 21) // n)
    for b0 in range(0, batch, blk):
        b1 = min(batch, b0 + blk)
        acc = noise[b0:b1].astype(np.complex128)
        for k in range(freqs.shape[1]):
            acc += t[(freqs[b0:b1, k, None] * j[None, :]) % n]
        out[b0:b1] = acc
    return out, freqs


def ragged_exponents(count: int, seed: int = DEFAULT_SEED, lo: int = 5, hi: int = 10):
    """``[count, 2]`` int array of (log2 nx, log2 ny), i.i.d. uniform on {lo..hi}."""
    rng = _rng(seed)
    return rng.integers(lo, hi + 1, size=(int(count), 2), dtype=np.int64)


def ragged_batch(count: int, seed: int = DEFAULT_SEED, lo: int = 5, hi: int = 10):
    """Ragged batch: shapes from :func:`ragged_exponents` and one packed
    complex64 buffer with each instance's ``[ny][nx]`` array stored back to back
    (re/im U[-1,1)).  Returns ``(nx, ny, offsets, packed)``; ``offsets[i]`` is
    the element offset of instance ``i`` in ``packed``.
    """
    e = ragged_exponents(count, seed=seed, lo=lo, hi=hi)
    nx = (1 << e[:, 0]).astype(np.int64)
    ny = (1 << e[:, 1]).astype(np.int64)
    sizes = nx * ny
    offsets = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    packed = uniform_complex((int(offsets[-1]),), seed=seed + 1)
    return nx, ny, offsets[:-1].copy(), packed
