"""The reference gradient of the differentiation workload, pinned on the CPU.

For L(x) = sum w * |F x|^2 (F the unnormalised forward 2D DFT, w >= 0 real),
PyTorch's gradient convention for a real loss of complex x is
dL/dRe(x) + i dL/dIm(x) = 2 F^H (w (.) F x) = 2 N IFFT2(w (.) FFT2(x)).
This file checks that closed form, evaluated with the FP64 oracle, against
FP64 central finite differences (h = 1e-6) of L itself on 64 x 64 -- so the
GPU gradient tests compare against a formula that is pinned independently.
"""
import numpy as np

import oracle
import synth


def loss(x, w):
    X = oracle.fft2d(x, dir=-1, threads=4)
    return np.sum(w * np.abs(X) ** 2, axis=(-2, -1))


def analytic_grad(x, w):
    X = oracle.fft2d(x, dir=-1, threads=4)
    return 2.0 * oracle.fft2d(w * X, dir=1, threads=4)


def test_gradient_formula_matches_central_differences_64x64():
    n = 64
    x = synth.uniform_complex((n, n), seed=2506).astype(np.complex128)
    w = synth.mask((n, n), seed=2507).astype(np.float64)
    h = 1e-6
    g_fd = np.zeros((n * n,), np.complex128)
    flat = x.reshape(-1)
    chunk = 512
    for part, unit in ((0, 1.0), (1, 1j)):
        for s in range(0, n * n, chunk):
            idx = np.arange(s, min(n * n, s + chunk))
            plus = np.repeat(flat[None, :], idx.size, axis=0)
            minus = plus.copy()
            plus[np.arange(idx.size), idx] += h * unit
            minus[np.arange(idx.size), idx] -= h * unit
            d = (loss(plus.reshape(-1, n, n), w) - loss(minus.reshape(-1, n, n), w)) / (2 * h)
            if part == 0:
                g_fd[idx] += d
            else:
                g_fd[idx] += 1j * d
    g = analytic_grad(x, w).reshape(-1)
    rel = np.max(np.abs(g_fd - g)) / np.max(np.abs(g))
    assert rel < 1e-6, rel


def test_gradient_formula_special_case_unit_weights():
    # w = 1: L = sum |F x|^2 = N sum |x|^2 (Parseval), so the gradient is 2 N x
    n = 32
    x = synth.uniform_complex((2, n, n), seed=3).astype(np.complex128)
    g = analytic_grad(x, np.ones((n, n)))
    assert np.max(np.abs(g - 2 * n * n * x)) < 1e-10 * n * n
