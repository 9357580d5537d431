"""Pins for the FP64 oracle: things the mathematics fixes, independent of the
oracle's own code.

* the O(N^2) definition (brute force, integer-reduced phases) on every small size;
* hand-derived DFTs of tiny inputs (tests/golden/dft_small.json);
* closed forms: delta -> constant, constant -> N*delta, unit exponential -> spike;
* invariants: linearity, Parseval, inverse(forward(x)) = N*x, shift theorem,
  Hermitian symmetry of real input, 2D = rows then columns;
* a library routine in the one case it reduces to (numpy.fft in complex128);
* mutation: every deliberately broken oracle build fails at least one pin.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dft_small.json")
POW2 = [1, 2, 4, 8, 16, 32, 64]


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)


def _rand(shape, seed):
    return synth.uniform_complex(shape, seed=seed).astype(np.complex128)


# ---------------------------------------------------------------------------
# Pin functions: each returns a list of failure strings for the given oracle
# library, so the same pins run against the real build and against mutants.
# ---------------------------------------------------------------------------

def pin_bruteforce_1d(lib):
    bad = []
    for n in POW2:
        x = _rand((3, n), 100 + n)
        for d in (-1, 1):
            got = oracle.fft1d_batch(x, dir=d, lib=lib)
            for r in range(3):
                ref = oracle.dft1d_brute(x[r], dir=d, lib=lib)
                if _rel(got[r], ref) > 1e-13:
                    bad.append(f"1d n={n} dir={d} row={r}")
    return bad


def pin_bruteforce_2d(lib):
    bad = []
    for ny in [1, 2, 4, 8, 16]:
        for nx in [1, 2, 4, 8, 16]:
            x = _rand((2, ny, nx), 7 * nx + ny)
            for d in (-1, 1):
                got = oracle.fft2d(x, dir=d, lib=lib)
                for b in range(2):
                    ref = oracle.dft2d_brute(x[b], dir=d, lib=lib)
                    if _rel(got[b], ref) > 1e-13:
                        bad.append(f"2d {ny}x{nx} dir={d} b={b}")
    return bad


def pin_golden(lib):
    bad = []
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        x = np.array([complex(a, b) for a, b in c["x"]]).reshape(c["shape"])
        X = np.array([complex(a, b) for a, b in c["X"]]).reshape(c["shape"])
        d = c["dir"]
        if len(c["shape"]) == 1:
            outs = [oracle.fft1d_batch(x, dir=d, lib=lib), oracle.dft1d_brute(x, dir=d, lib=lib)]
        else:
            outs = [oracle.fft2d(x, dir=d, lib=lib), oracle.dft2d_brute(x, dir=d, lib=lib)]
        for k, o in enumerate(outs):
            if np.abs(o - X).max() > 1e-14 * max(1.0, np.abs(X).max()):
                bad.append(f"golden {c['name']} ({['fft', 'brute'][k]})")
    return bad


def pin_closed_forms(lib):
    bad = []
    for ny, nx in [(1, 64), (8, 32), (32, 16), (64, 64), (2, 1024)]:
        N = nx * ny
        delta = np.zeros((ny, nx), np.complex128)
        delta[0, 0] = 1.0
        for d in (-1, 1):
            if np.abs(oracle.fft2d(delta, dir=d, lib=lib) - 1.0).max() > 1e-14:
                bad.append(f"delta {ny}x{nx} dir={d}")
        ones = np.ones((ny, nx), np.complex128)
        spike = np.zeros((ny, nx), np.complex128)
        spike[0, 0] = N
        if np.abs(oracle.fft2d(ones, lib=lib) - spike).max() > 1e-12 * N:
            bad.append(f"const {ny}x{nx}")
        rng = np.random.default_rng(N)
        for _ in range(3):
            fy, fx = int(rng.integers(ny)), int(rng.integers(nx))
            yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
            phase = ((fx * xx) % nx) / nx + ((fy * yy) % ny) / ny
            e = np.exp(2j * np.pi * phase)
            want = np.zeros((ny, nx), np.complex128)
            want[fy, fx] = N
            if np.abs(oracle.fft2d(e, dir=-1, lib=lib) - want).max() > 1e-12 * N:
                bad.append(f"exp spike {ny}x{nx} f=({fy},{fx}) fwd")
            # the inverse maps the conjugate exponential to the same spike
            if np.abs(oracle.fft2d(np.conj(e), dir=1, lib=lib) - want).max() > 1e-12 * N:
                bad.append(f"exp spike {ny}x{nx} f=({fy},{fx}) inv")
    return bad


def pin_invariants(lib):
    bad = []
    for ny, nx in [(16, 8), (64, 128), (256, 32), (4, 512)]:
        N = nx * ny
        x = _rand((ny, nx), 31 + N)
        z = _rand((ny, nx), 37 + N)
        X, Z = oracle.fft2d(x, lib=lib), oracle.fft2d(z, lib=lib)
        a, b = 0.75 - 0.5j, -1.25 + 2j
        if _rel(oracle.fft2d(a * x + b * z, lib=lib), a * X + b * Z) > 1e-14:
            bad.append(f"linearity {ny}x{nx}")
        if abs(np.sum(np.abs(X) ** 2) - N * np.sum(np.abs(x) ** 2)) > 1e-12 * N * np.sum(np.abs(x) ** 2):
            bad.append(f"parseval {ny}x{nx}")
        if _rel(oracle.fft2d(X, dir=1, lib=lib), N * x) > 1e-14:
            bad.append(f"inverse {ny}x{nx}")
        sy, sx = 3 % ny, 5 % nx
        xs = np.roll(x, shift=(sy, sx), axis=(0, 1))
        ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ph = np.exp(-2j * np.pi * (((ky * sy) % ny) / ny + ((kx * sx) % nx) / nx))
        if _rel(oracle.fft2d(xs, lib=lib), ph * X) > 1e-13:
            bad.append(f"shift {ny}x{nx}")
        r = x.real.astype(np.complex128)
        R = oracle.fft2d(r, lib=lib)
        mirror = np.conj(R[(-ky) % ny, (-kx) % nx])
        if _rel(R, mirror) > 1e-14:
            bad.append(f"hermitian {ny}x{nx}")
        # 2D = 1D along rows, then 1D along columns
        rows = oracle.fft1d_batch(x, lib=lib)
        cols = oracle.fft1d_batch(rows.T.copy(), lib=lib).T
        if _rel(X, cols) > 1e-14:
            bad.append(f"separable {ny}x{nx}")
    return bad


def pin_library(lib):
    bad = []
    for ny, nx in [(8, 8), (32, 64), (128, 16), (256, 256)]:
        x = _rand((2, ny, nx), nx + 3 * ny)
        if _rel(oracle.fft2d(x, lib=lib), np.fft.fft2(x)) > 1e-14:
            bad.append(f"numpy fwd {ny}x{nx}")
        if _rel(oracle.fft2d(x, dir=1, lib=lib), np.fft.ifft2(x) * nx * ny) > 1e-14:
            bad.append(f"numpy inv {ny}x{nx}")
    return bad


def pin_sampled(lib):
    bad = []
    for ny, nx in [(16, 32), (64, 8), (128, 128)]:
        x = _rand((ny, nx), 5 * nx + ny)
        for d in (-1, 1):
            X = oracle.fft2d(x, dir=d, lib=lib)
            ky = np.array([0, 1, ny // 2, ny - 1])
            kx = np.array([0, nx // 3, nx - 1])
            if _rel(oracle.fft2d_rows(x, ky, dir=d, lib=lib), X[ky]) > 1e-13:
                bad.append(f"rows {ny}x{nx} dir={d}")
            if _rel(oracle.fft2d_cols(x, kx, dir=d, lib=lib), X[:, kx].T) > 1e-13:
                bad.append(f"cols {ny}x{nx} dir={d}")
    return bad


def pin_bins(lib):
    """Single bins of long 1D transforms: the definition per bin against the
    recursive transform (two independent evaluations), and a closed form."""
    bad = []
    for n in [64, 4096, 1 << 16]:
        x = _rand((n,), 11 + n)
        bins = np.array(sorted({0, 1, 3, n // 2, n // 2 + 1, n - 1, (7 * n) // 11}))
        for d in (-1, 1):
            X = oracle.fft1d_batch(x, dir=d, lib=lib)
            if _rel(oracle.dft1d_bins(x, bins, dir=d, threads=2, lib=lib), X[bins]) > 1e-12:
                bad.append(f"bins n={n} dir={d}")
    n, f = 1 << 20, 12345
    e = np.exp(2j * np.pi * ((f * np.arange(n)) % n) / n)
    got = oracle.dft1d_bins(e, [f, f + 1, 0], dir=-1, threads=3, lib=lib)
    if np.abs(got - np.array([n, 0, 0])).max() > 1e-9 * n:
        bad.append("bins exp spike")
    return bad


def pin_any_length(lib):
    """Any-length recursion: the definition for every n <= 64 and for
    composite, prime and prime-power lengths; the radix-2 recursion at powers
    of two; a closed form; Parseval and the round trip; 2D against the 2D
    definition."""
    bad = []
    for n in list(range(1, 65)) + [96, 100, 127, 210, 243, 625, 1001]:
        x = _rand((2, n), 500 + n)
        for d in (-1, 1):
            got = oracle.fft1d_any(x, dir=d, lib=lib)
            for r in range(2):
                if _rel(got[r], oracle.dft1d_brute(x[r], dir=d, lib=lib)) > 1e-13:
                    bad.append(f"any n={n} dir={d}")
    for n in (256, 4096):
        x = _rand((n,), 7 * n)
        if _rel(oracle.fft1d_any(x, lib=lib), oracle.fft1d_batch(x, lib=lib)) > 1e-13:
            bad.append(f"any vs radix-2 n={n}")
    n, f = 3000, 1234
    e = np.exp(2j * np.pi * ((f * np.arange(n)) % n) / n)
    want = np.zeros(n, np.complex128)
    want[f] = n
    if np.abs(oracle.fft1d_any(e, lib=lib) - want).max() > 1e-10 * n:
        bad.append("any exp spike")
    n = 3 * 5 * 7 * 11
    x = _rand((n,), 99)
    X = oracle.fft1d_any(x, lib=lib)
    if abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) > 1e-12 * n * np.sum(np.abs(x) ** 2):
        bad.append("any parseval")
    if _rel(oracle.fft1d_any(X, dir=1, lib=lib), n * x) > 1e-13:
        bad.append("any roundtrip")
    for ny, nx in [(3, 5), (6, 10), (12, 7), (15, 15), (1, 9), (11, 1)]:
        x = _rand((ny, nx), 3 * nx + ny)
        for d in (-1, 1):
            if _rel(oracle.fft2d_any(x, dir=d, lib=lib), oracle.dft2d_brute(x, dir=d, lib=lib)) > 1e-13:
                bad.append(f"any 2d {ny}x{nx} dir={d}")
    x = _rand((2, 32, 64), 17)
    if _rel(oracle.fft2d_any(x, lib=lib), oracle.fft2d(x, lib=lib)) > 1e-13:
        bad.append("any 2d vs radix-2")
    return bad


PINS = [pin_bruteforce_1d, pin_bruteforce_2d, pin_golden, pin_closed_forms,
        pin_invariants, pin_library, pin_sampled, pin_bins, pin_any_length]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_pin(pin):
    bad = pin(oracle.load())
    assert not bad, bad


def test_brute_force_itself_matches_golden():
    # the brute force is the definition; pin it to hand-derived values too
    assert not pin_golden(oracle.load())


def test_threads_do_not_change_results():
    x = _rand((4, 64, 128), 9)
    a = oracle.fft2d(x, threads=1)
    b = oracle.fft2d(x, threads=4)
    assert np.array_equal(a, b)


def test_bad_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.fft1d_batch(np.zeros(6, np.complex64))
    with pytest.raises(ValueError):
        oracle.fft2d(np.zeros((3, 4), np.complex64))


# Each mutant plants one plausible mistake in oracle.c (see ORACLE_MUTANT):
# 1 twiddle sign, 2 dropped term, 3 off-by-one twiddle index, 4 transposed
# length in the column pass, 5 dropped column pass, 6 conjugated input,
# 7 brute-force sign, 8 neighbouring bin in the per-bin definition, 9 the
# any-length combining phase reduced modulo the wrong length.  Every one must
# fail at least one pin.
@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_pins_catch_mutant(mutant):
    lib = oracle.load(mutant=mutant)
    failures = []
    for pin in PINS:
        try:
            failures += pin(lib)
        except Exception as e:  # a crash counts as caught too
            failures.append(f"{pin.__name__}: {e!r}")
    assert failures, f"mutant {mutant} passed every pin"
