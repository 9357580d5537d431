"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol include/gb300fft.h declares, and its host-side logic (argument
validation, error strings, stage schedules) behaves -- no GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from tests.helpers import digit_reversal

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gb300fft.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2506_15437_gb300 import build
    build.build()
    from paper_2506_15437_gb300 import _native
    return _native.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fft_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_core_abi():
    names = declared_functions()
    for n in ["fft_plan_create", "fft_execute", "fft_backward", "fft_plan_destroy",
              "fft_plan_create_ragged", "fft_execute_ragged", "fft_plan_status",
              "fft_debug_reorder_map"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in gb300fft.h but not exported"


def test_binding_covers_header():
    from paper_2506_15437_gb300 import _native
    bound = {n for n, _, _ in _native.SIGNATURES}
    assert set(declared_functions()) == bound


def test_error_strings(lib):
    for code in [0, -1, -2, -3, -4, -5, -6, 12345]:
        s = lib.fft_error_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert b"timed out" in lib.fft_error_string(-6)


@pytest.mark.parametrize("nx,ny,batch", [(0, 3, 1), (3, 0, 1), (0, 8, 1), (8, 8, 0),
                                         (131072, 2, 1), (2, 131072, 1), (-4, 4, 1),
                                         (1 << 27, 1, 1), (1, 1 << 27, 1), (3 << 23, 1, 1),
                                         (70000, 3, 1), (1 << 26, 1, 64)])
def test_invalid_sizes_rejected_without_touching_the_gpu(lib, nx, ny, batch):
    assert lib.fft_plan_create(nx, ny, batch, -1, 0) is None
    assert lib.fft_last_error() == -1


def test_long_1d_and_any_size_are_fp32_only(lib):
    # the four-step path (1D lengths above 8192), sizes that are not
    # powers of two and 2D axes above 8192 (planned axis by axis) have no
    # split-FP16 form; the request is refused before any device call
    assert lib.fft_plan_create(1 << 16, 1, 1, -1, 1) is None
    assert lib.fft_last_error() == -5
    assert lib.fft_plan_create(1000, 3, 1, -1, 1) is None
    assert lib.fft_last_error() == -5
    assert lib.fft_plan_create(16384, 2, 1, -1, 1) is None  # 2D axis above 8192: axis by axis
    assert lib.fft_last_error() == -5


def test_invalid_direction_and_precision(lib):
    assert lib.fft_plan_create(8, 8, 1, 0, 0) is None
    assert lib.fft_last_error() == -2
    assert lib.fft_plan_create(8, 8, 1, -1, 7) is None
    assert lib.fft_last_error() == -2


def test_null_plan_calls(lib):
    assert lib.fft_plan_destroy(None) == 0
    assert lib.fft_execute(None, None, None, None) == -2
    assert lib.fft_backward(None, None, None, None) == -2
    assert lib.fft_plan_status(None, None) == -2
    off = ctypes.c_longlong(0)
    assert lib.fft_ragged_offset(None, 0, ctypes.byref(off)) < 0
    # the fused differentiation form: a NULL plan is an argument error
    assert lib.fft_weighted_power_adjoint_parts(None) == -2
    assert lib.fft_weighted_power_adjoint(None, None, None, None, None, None) == -2
    assert lib.fft_backward_rows_scaled(None, None, None, 1.0, None, None) == -2


def test_last_cuda_error_text(lib):
    """A readable string whatever state the runtime is in (here, without
    a GPU, whatever the runtime reports for that)."""
    t = lib.fft_debug_last_cuda_error()
    assert isinstance(t, bytes) and len(t) > 0


def test_ragged_rejects_out_of_range_sizes(lib):
    nx = (ctypes.c_int * 2)(32, 2048)
    ny = (ctypes.c_int * 2)(32, 32)
    assert lib.fft_plan_create_ragged(2, nx, ny, -1, 0) is None
    assert lib.fft_last_error() in (-1, -5)
    assert lib.fft_plan_create_ragged(0, nx, ny, -1, 0) is None


@pytest.mark.parametrize("axis", [0, 1])
def test_stage_schedules(lib, axis):
    buf = (ctypes.c_int * 16)()
    for L in range(0, 14):
        n = 1 << L
        k = lib.fft_debug_radices(n, axis, buf)
        assert k >= 1
        rad = [buf[i] for i in range(k)]
        assert int(np.prod(rad)) == n
        assert all(r & (r - 1) == 0 for r in rad)
        assert all(r <= 32 for r in rad)
    assert lib.fft_debug_radices(12, axis, buf) < 0


def _smooth13(n):
    for p in (2, 3, 5, 7, 11, 13):
        while n % p == 0:
            n //= p
    return n == 1


MIXED_RADICES = set(range(2, 17))


def _fewest_stages(limit):
    """fewest[m]: the fewest factors from MIXED_RADICES whose product is m
    (dynamic programming over m; None where m has another prime factor)."""
    fewest = [None] * (limit + 1)
    fewest[1] = 0
    for m in range(2, limit + 1):
        c = [fewest[m // r] for r in MIXED_RADICES if m % r == 0 and fewest[m // r] is not None]
        fewest[m] = 1 + min(c) if c else None
    return fewest


def test_mixed_radix_schedules(lib):
    """Host-side mixed-radix planning, without a GPU: every length up to
    3000 and the longest one-CTA lengths factor into the compiled radices
    with product n and no more stages than the fewest possible (found here
    by brute force); the greedy schedules of the tuned lengths are kept;
    other lengths are refused."""
    buf = (ctypes.c_int * 16)()
    n1, n2 = ctypes.c_int(), ctypes.c_int()
    fewest = _fewest_stages(14336)
    for n in list(range(2, 3001)) + [14336, 14335, 12288, 10000]:
        k = lib.fft_debug_mixed_plan(n, buf, ctypes.byref(n1), ctypes.byref(n2))
        if not _smooth13(n):
            assert k == -1, n
            continue
        assert 1 <= k <= 16 and n1.value == 0 and n2.value == 0, n
        rad = [buf[i] for i in range(k)]
        assert int(np.prod(rad)) == n, (n, rad)
        assert set(rad) <= MIXED_RADICES, (n, rad)
        assert k == fewest[n], (n, rad, fewest[n])
    expect = {3000: [8, 15, 5, 5], 1080: [8, 15, 9], 1920: [16, 8, 15], 14336: [16, 16, 8, 7],
              1000: [10, 10, 10], 10000: [10, 10, 10, 10], 96: [16, 6], 1728: [16, 12, 9], 210: [15, 14],
              4095: [15, 3, 7, 13], 1001: [7, 11, 13], 143: [11, 13], 2197: [13, 13, 13]}
    for n, rad in expect.items():
        k = lib.fft_debug_mixed_plan(n, buf, ctypes.byref(n1), ctypes.byref(n2))
        assert [buf[i] for i in range(k)] == rad, n


def test_mixed_fourstep_splits(lib):
    """Smooth lengths beyond one CTA: n = n1 n2, both mixed-radix lengths
    (<= 14336), with n2 the divisor closest to sqrt(n) in log scale."""
    buf = (ctypes.c_int * 16)()
    n1, n2 = ctypes.c_int(), ctypes.c_int()
    for n in [15360, 20000, 10 ** 6, 3 << 20, 6 ** 9, 5 ** 10, 7 ** 8, 14337 * 0 + 16384 * 3]:
        assert lib.fft_debug_mixed_plan(n, buf, ctypes.byref(n1), ctypes.byref(n2)) == 0, n
        a, b = n1.value, n2.value
        assert a * b == n and max(a, b) <= 14336 and _smooth13(a) and _smooth13(b), (n, a, b)
        divs = [d for d in range(2, 14337) if n % d == 0 and n // d <= 14336]
        best = min(divs, key=lambda d: abs(np.log(d) - 0.5 * np.log(n)))
        assert abs(np.log(b) - 0.5 * np.log(n)) <= abs(np.log(best) - 0.5 * np.log(n)) + 1e-12, (n, b, best)
    for n in (17 * 3000, 1 << 25, 0, 1):
        assert lib.fft_debug_mixed_plan(n, buf, ctypes.byref(n1), ctypes.byref(n2)) < 0, n


def test_compile_time_roots_are_correctly_rounded(lib):
    """The constants of the composite-radix DFTs (cos and sin of 2 pi m / R
    evaluated by the compiler): equal to the float nearest the exact value
    for every R <= 128 and m < R, and exactly 0 or +-1 on the axes.  The
    reference is mpmath-free: FP64 libm values, accepted only where the
    float rounding is unambiguous (|x - float midpoint| well above 1e-15)."""
    import math
    c, s = ctypes.c_float(), ctypes.c_float()
    checked = 0
    for R in range(1, 129):
        for m in range(R):
            assert lib.fft_debug_root(m, R, ctypes.byref(c), ctypes.byref(s)) == 0
            for got, want in ((c.value, math.cos(2 * math.pi * m / R)), (s.value, math.sin(2 * math.pi * m / R))):
                if (4 * m) % R == 0:  # on an axis: exact
                    want = float(round(want))
                    assert got == want, (m, R, got, want)
                    continue
                f = float(np.float32(want))
                # skip the rare values within 1e-15 of a rounding midpoint
                nxt = float(np.nextafter(np.float32(f), np.float32(np.inf if want > f else -np.inf)))
                if abs(abs(want - f) - abs(nxt - f) / 2) < 1e-15:
                    continue
                assert got == f, (m, R, got, f)
                checked += 1
    assert checked > 10000
    assert lib.fft_debug_root(1, 0, ctypes.byref(c), ctypes.byref(s)) < 0


def test_digit_reversal_helper_is_a_bijection_and_bit_reversal_for_radix2():
    for L in range(1, 12):
        n = 1 << L
        m = digit_reversal(n, [2] * L)
        assert sorted(m) == list(range(n))
        br = [int(format(i, f"0{L}b")[::-1], 2) for i in range(n)]
        assert list(m) == br


def test_product_path_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    import paper_2506_15437_gb300 as g
    x = torch.zeros(8, 8, dtype=torch.complex64)
    with pytest.raises((ValueError, RuntimeError)):
        g.fft2(x)
