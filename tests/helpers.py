"""Shared test utilities: error metric, tolerances, digit reversal."""
import math
import os

import numpy as np

ORACLE_THREADS = max(1, min(16, os.cpu_count() or 1))


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.complex128).ravel()
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def worst_rel_l2(got, ref, per) -> float:
    """Worst relative L2 error over transforms of `per` elements each."""
    got = np.asarray(got).reshape(-1, per)
    ref = np.asarray(ref).reshape(-1, per)
    return max(rel_l2(g, r) for g, r in zip(got, ref))


def tol_fp32(N: int) -> float:
    """Plain FP32 path bound: rel L2 <= 2e-7 * log2(N), N points per transform."""
    return 2e-7 * max(1.0, math.log2(N))


def tol_split_tc(N: int) -> float:
    return 1e-6 * max(1.0, math.log2(N))


def digit_reversal(n: int, radices) -> np.ndarray:
    """map[i] for the mixed-radix digit reversal: write i with digits d_0 (radix
    R_0, most significant) ... d_{S-1}, then map[i] = d_0 + d_1 R_0 + d_2 R_0 R_1 + ..."""
    i = np.arange(n, dtype=np.int64)
    out = np.zeros(n, dtype=np.int64)
    w = n
    mult = 1
    rem = i.copy()
    for R in radices:
        w //= R
        d = rem // w
        rem = rem % w
        out += d * mult
        mult *= R
    return out


def bluestein_m(n: int) -> int:
    """Power-of-two length of the circular convolution for a length-n axis."""
    m = 1
    while m < 2 * n - 1:
        m <<= 1
    return m


MIXED_MAX_N = 14336  # longest mixed-radix length (two float2 buffers in one CTA's shared memory)


def odd_factors(n: int) -> int:
    """Number of prime factors 3, 5, 7, 11, 13 of n (with multiplicity) if n
    is 13-smooth, else -1."""
    k = 0
    for p in (3, 5, 7, 11, 13):
        while n % p == 0:
            n //= p
            k += 1
    while n % 2 == 0:
        n //= 2
    return k if n == 1 else -1


def mixed_eligible(n: int) -> bool:
    """Lengths the mixed-radix kernel takes: 13-smooth, not a power of two,
    at most MIXED_MAX_N."""
    return n & (n - 1) != 0 and n <= MIXED_MAX_N and odd_factors(n) >= 0


def tol_bluestein_axis(n: int) -> float:
    """Bluestein: two transforms of length M = bluestein_m(n), the filter
    transform (a third one, computed once in FP32) and three roundings by
    unit-modulus factors, so 2e-7 * (3 * log2 M + 3)."""
    return 2e-7 * (3 * math.log2(bluestein_m(n)) + 3)


def tol_mixed_axis(n: int) -> float:
    """Mixed radix (one pass or the four-step form): the plain path's bound
    2e-7 * log2 n, with log2 n the radix-2-equivalent depth of the length."""
    return 2e-7 * math.log2(n)


def mixed_fourstep_eligible(n: int) -> bool:
    """Longer 13-smooth lengths (not powers of two): two mixed-radix passes
    of a four-step split (every such length up to 2^24 has a divisor
    between n / MIXED_MAX_N and MIXED_MAX_N)."""
    return n & (n - 1) != 0 and MIXED_MAX_N < n <= (1 << 24) and odd_factors(n) >= 0


def tol_any_axis(n: int, mixed: bool = True) -> float:
    """FP32 bound for one axis of any length: a power of two is the plain
    path (2e-7 * log2 n); a 13-smooth length up to MIXED_MAX_N the mixed-radix
    kernel and a longer one its four-step form, both held to the same
    2e-7 * log2 n, unless `mixed` is False (the plan was made with it switched
    off); any other length Bluestein."""
    if n & (n - 1) == 0:
        return 2e-7 * max(1.0, math.log2(n))
    if mixed and (mixed_eligible(n) or mixed_fourstep_eligible(n)):
        return tol_mixed_axis(n)
    return tol_bluestein_axis(n)


def tol_any(nx: int, ny: int, mixed: bool = True) -> float:
    """Errors of the two axes add (a transpose is exact)."""
    return tol_any_axis(nx, mixed) + (tol_any_axis(ny, mixed) if ny > 1 else 0.0)
