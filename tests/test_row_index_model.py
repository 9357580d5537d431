"""CPU model of the row-pass kernel's index arithmetic (no GPU).

For every row kernel the library compiles -- length n, elements per thread
E, column pre-split P -- the launch shape comes from the library itself
(fft_debug_row_variant: threads, rows per CTA, shared-memory elements per
row, stage radices).  The model then walks every CTA, loop iteration and
thread of a launch the way the kernel does and checks, for a set of row
counts, slice heights, persistent grids, L2-prefetch distances and
streaming/planar store orders:

* every global load (both input rows of a pre-split pair), every L2 bulk
  prefetch range and every pre-split twiddle index lies inside its buffer;
* every row's stage-0 loads read each element exactly once;
* the stores of a launch hit each output element exactly once;
* each shared-memory exchange writes and reads stay inside the row's padded
  span, and each stage's writes are a bijection onto the padded images of
  0..n-1 (no two threads write one word).

The model restates the kernel's address formulas (Stockham stage s of radix
R and span Ns: butterfly j reads j + r n/R and writes (j - m) R + m + k Ns
with m = j mod Ns; Section 2.2's butterflies in self-sorting order), so it
checks bounds and bijectivity of those formulas for every compiled shape.
"""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2506_15437_gb300 import build
    build.build()
    from paper_2506_15437_gb300 import _native
    return _native.load()


def variant(lib, n, e, split):
    info = (ctypes.c_int * 20)()
    rc = lib.fft_debug_row_variant(n, e, split, info)
    if rc != 0:
        return None
    S = info[3]
    return dict(threads=info[0], rows=info[1], smem=info[2], radices=[info[4 + k] for k in range(S)])


def pad_shift(E):
    return 6 if E >= 64 else 5 if E >= 32 else 4


def pad_shift1(E):
    return 4 if E == 32 else pad_shift(E)


def check_shared(n, E, rad, smem_elems):
    """Stage exchanges of one row (W = 1, c = 0)."""
    S = len(rad)
    assert all(r == E for r in rad[1:]), rad
    R0 = rad[0]
    T = n // E
    tt = np.arange(T)
    span = 1
    for s in range(1, S):
        Rp = R0 if s == 1 else E
        Nsp = span  # span of stage s - 1
        sh = pad_shift1(E) if s == 1 else pad_shift(E)
        pad = lambda f: f + (f >> sh)  # noqa: E731
        # writes of stage s - 1's outputs
        b = np.arange(E // Rp)
        j = tt[:, None] + b[None, :] * T
        m = j & (Nsp - 1)
        k = np.arange(Rp)
        f = ((j - m)[..., None] * Rp + m[..., None] + k[None, None, :] * Nsp).ravel()
        assert np.array_equal(np.sort(f), np.arange(n)), ("stage write not a bijection", n, E, s)
        w = pad(f)
        assert w.min() >= 0 and w.max() < smem_elems, ("write out of span", n, E, s)
        assert np.unique(w).size == n
        # reads of stage s's operands
        r = np.arange(E)
        fr = (tt[:, None] + r[None, :] * T).ravel()
        assert np.array_equal(np.sort(fr), np.arange(n))
        rr = pad(fr)
        assert rr.min() >= 0 and rr.max() < smem_elems, ("read out of span", n, E, s)
        span *= Rp


def model_launch(n, E, rows_per_cta, rad, P, ny, batch, grid, pf, perm_t=0, perm_g=1, planar=0):
    """Global addresses of one row-pass launch over nrows = ny * batch rows."""
    R0 = rad[0]
    RL = rad[-1] if len(rad) > 1 else R0
    T = n // E
    ROWS = rows_per_cta
    nrows = ny * batch
    Q = ny // P
    total = nrows * n
    tt = np.arange(T)
    # stage-0 element indices of one row, as the threads load them
    b = np.arange(E // R0)
    r = np.arange(R0)
    i_load = (tt[:, None, None] + b[None, :, None] * T + r[None, None, :] * (n // R0)).ravel()
    assert np.array_equal(np.sort(i_load), np.arange(n))
    # natural-order output positions of the last stage
    b = np.arange(E // RL)
    k = np.arange(RL)
    i_store = (tt[:, None, None] + b[None, :, None] * T + k[None, None, :] * (n // RL)).ravel()
    assert np.array_equal(np.sort(i_store), np.arange(n))

    def in_row(row, p):
        if P == 1:
            return row
        bb, y = divmod(row, ny)
        return bb * ny + y // P + Q * p

    written = np.zeros(total, dtype=np.int32)
    step = grid * ROWS
    groups = (nrows + ROWS - 1) // ROWS
    assert 1 <= grid <= groups
    for cta in range(grid):
        # start-up prefetches (pf > 1)
        for d in range(1, pf):
            nb = cta * ROWS + d * step
            if nb >= nrows:
                break
            for gg in range(ROWS):
                if nb + gg >= nrows:
                    break
                for p in range(P):
                    a = in_row(nb + gg, p) * n
                    assert 0 <= a and a + n <= total
        base = cta * ROWS
        while base < nrows:
            nb = base + (pf if pf > 0 else 1) * step
            if pf > 0 and nb < nrows:
                if P == 1:
                    cnt = min(nrows - nb, ROWS)
                    assert 0 <= nb * n and (nb + cnt) * n <= total
                else:
                    for gg in range(ROWS):
                        if nb + gg >= nrows:
                            break
                        for p in range(P):
                            a = in_row(nb + gg, p) * n
                            assert 0 <= a and a + n <= total
            for g in range(ROWS):
                row = base + g
                if row >= nrows:
                    continue
                for p in range(P):
                    ir = in_row(row, p)
                    assert 0 <= ir < nrows, (row, p, ir)
                if P > 1:
                    y = row % ny
                    kp, q = y % P, y // P
                    assert 0 <= q * kp < ny  # the pre-split twiddle table has ny entries
                orow = row
                if perm_t or planar:
                    bb, y = divmod(row, ny)
                    i, kq = y // P, y % P
                    pos = i
                    if perm_t:
                        j, rr = i & (perm_t - 1), i // perm_t
                        pos = (j // perm_g) * perm_g * (Q // perm_t) + rr * perm_g + (j & (perm_g - 1))
                    orow = bb * ny + (kq * Q + pos if planar else kq + P * pos)
                assert 0 <= orow < nrows, (row, orow)
                written[orow * n + i_store] += 1
            base += step
    assert written.min() == 1 and written.max() == 1, "stores are not a bijection onto the output"


def compiled_variants(lib):
    out = []
    for L in range(1, 14):
        n = 1 << L
        for e in (8, 16, 32):
            for split in (1, 2):
                v = variant(lib, n, e, split)
                if v is not None:
                    out.append((n, min(e, n), split, v))
    return out


def test_registry_shapes(lib):
    vs = compiled_variants(lib)
    keys = {(n, e, s) for n, e, s, _ in vs}
    # the E = 32 pre-split kernel exists for 8192-point rows only
    assert (8192, 32, 2) in keys
    for n in (1024, 2048, 4096):
        assert (n, 32, 2) not in keys
        assert (n, 32, 1) in keys
    for n, e, s, v in vs:
        T = n // e
        assert v["threads"] == v["rows"] * T, (n, e, s, v)
        assert int(np.prod(v["radices"])) == n
        assert v["radices"][0] <= e


@pytest.mark.parametrize("L", range(1, 14))
def test_shared_memory_exchanges_in_span(lib, L):
    n = 1 << L
    for e in (8, 16, 32):
        v = variant(lib, n, e, 1)
        if v is None:
            continue
        E = min(e, n)
        if len(v["radices"]) > 1:
            check_shared(n, E, v["radices"], v["smem"])


@pytest.mark.parametrize("L", range(1, 14))
def test_global_indices_in_bounds(lib, L):
    n = 1 << L
    for e in (8, 16, 32):
        for split in (1, 2):
            v = variant(lib, n, e, split)
            if v is None:
                continue
            E = min(e, n)
            R = v["rows"]
            cases = []
            if split == 1:
                for nrows in sorted({1, max(1, R - 1), R, R + 1, 3 * R + 2}):
                    cases.append((nrows, 1))
            else:
                for ny in (4, 8, 2 * R + 2 if (2 * R + 2) % 2 == 0 else 2 * R + 4):
                    for batch in (1, 2, 3):
                        cases.append((ny, batch))
            for ny, batch in cases:
                nrows = ny * batch
                groups = (nrows + R - 1) // R
                for grid in sorted({1, min(3, groups), groups}):
                    for pf in (0, 1, 2):
                        model_launch(n, E, R, v["radices"], split, ny, batch, grid, pf)


@pytest.mark.parametrize("planar", [0, 1])
@pytest.mark.parametrize("perm", [0, 1])
def test_streaming_row_orders_in_bounds(lib, planar, perm):
    """The row orders the streaming column pass asks for (4096-point column
    blocks: 64 stage-0 butterflies, 8 per warp), with and without the
    pre-split, plain and planar."""
    for n, e, split in [(8192, 32, 2), (8192, 16, 2), (4096, 16, 1), (256, 16, 1), (256, 16, 2)]:
        v = variant(lib, n, e, split)
        assert v is not None
        ny = 4096 * split
        for batch in (1, 2):
            nrows = ny * batch
            groups = (nrows + v["rows"] - 1) // v["rows"]
            model_launch(n, min(e, n), v["rows"], v["radices"], split, ny, batch, min(304, groups), 1,
                         perm_t=64 if perm else 0, perm_g=8, planar=planar)


def test_removed_presplit_variant_model_at_the_failing_shape():
    """The pre-split E = 32 kernel of 4096-point rows (two rows per CTA; no
    longer compiled) on the 4096 x 512 x 2 plan where it raised an illegal
    address: the model of its arithmetic stays in bounds on every grid the
    plan could launch, so the fault is not explained by these formulas."""
    n, E, R = 4096, 32, 2
    rad = [4, 32, 32]
    smem = 4351  # Engine<4096, 32> padded elements per row
    check_shared(n, E, rad, smem)
    for grid in (1, 152, 304, 456, 512):
        for pf in (0, 1):
            model_launch(n, E, R, rad, 2, 512, 2, grid, pf)
