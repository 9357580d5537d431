"""CPU model of the split-FP16 tensor-core kernels' layouts and index maps.

The compiled constants come from the library (fft_debug_tc_layout, host
only, no device call); the checks below redo each kernel's address
arithmetic in numpy and check it on the CPU:
- every shared-memory access stays inside its span, and spans do not
  overlap;
- every bulk copy starts on a 16-byte boundary;
- the landing, exchange, ring, B-table, barrier and TMEM-slot regions are
  disjoint and fit the 227 KiB of one CTA;
- the named-barrier ids are distinct per thread set and below 16;
- TMEM columns stay within each group's share;
- the permuted row order the row kernels store for the streaming column
  pass is a bijection onto the block rows, and lands each warp's stage-0
  operands in one contiguous segment.
"""
import ctypes

import numpy as np
import pytest

SMEM_MAX = 232448 - 1024  # shared memory of one CTA (227 KiB) less 1 KiB static (status words, alignment)


@pytest.fixture(scope="module")
def lib():
    from paper_2506_15437_gb300 import build
    build.build()
    from paper_2506_15437_gb300 import _native as N
    return N.load()


def layout(lib, n, kind):
    a = (ctypes.c_longlong * 32)()
    assert lib.fft_debug_tc_layout(n, kind, a) == 0
    return list(a)


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
def test_pair_landing_kernel_layout(lib, n):
    threads, T, L, xe, buf, b_off, bar_off, smem, land = layout(lib, n, 0)[:9]
    assert T == n // 32 and threads == 512 and L * T == threads
    # the landed rows [L][n] and the L exchange spans (stride = exchange size)
    # both fit the buffer; the exchange of output h aliases landed rows only
    assert land == L * n * 8 <= buf and L * xe * 8 <= buf
    assert land < (1 << 20)  # one mbarrier transaction count
    assert b_off >= buf and b_off % 1024 == 0 and bar_off == b_off + 2 * 8192
    assert bar_off + 64 <= smem <= SMEM_MAX
    # pair units: input rows q .. q + L/2 - 1 and their partners land at
    # (i, L/2 + i); output h = (pair i = h // 2, kp = h % 2) reads both
    uq = L // 2
    for h in range(L):
        i = h // 2
        assert 0 <= i < uq and uq + i < L


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
def test_subunit_landing_kernel_layout(lib, n):
    (threads, T, L, xe, RS, U, K, span, buf, b_off, bar_off, slot_off,
     smem) = layout(lib, n, 1)[:13]
    assert T == n // 32 and threads == 512 and L * T == threads
    assert U == RS * T and U in (128, 256) and K * U == threads and K * RS == L
    # row spans: 16-byte multiples (bulk copy destinations), each holds a
    # landed row and the row's padded exchange, pairwise disjoint
    assert span % 2 == 0 and span >= n and span >= xe and L * span * 8 == buf
    starts = np.arange(L) * span
    assert np.all(starts[1:] >= starts[:-1] + xe)
    assert b_off >= buf and b_off % 1024 == 0 and bar_off == b_off + 2 * 8192
    assert slot_off == bar_off + 8 * (4 + K) and slot_off + 16 <= smem <= SMEM_MAX
    # thread t: row h = t // T, sub-unit k = t // U, which owns rows
    # k*RS .. k*RS + RS - 1 (the spans its lead thread lands)
    t = np.arange(threads)
    h, k = t // T, t // U
    assert np.all((h >= k * RS) & (h < (k + 1) * RS))
    # barrier ids: 0 the CTA, 1-4 the MMA groups (128 threads), rows 5 + h
    # (rows of 64 or more threads; 32-thread rows use the warp), sub-units
    # the group id (U = 128) or the row id (U = 256)
    group_ids = 1 + t // 128
    row_ids = 5 + h if T >= 64 else None
    sub_ids = group_ids if U == 128 else 5 + k
    assert group_ids.max() <= 15 and sub_ids.max() <= 15
    if row_ids is not None:
        assert row_ids.max() <= 15
        # one id, one thread set: rows never share an id with a group of
        # other threads
        for rid in np.unique(row_ids):
            members = set(t[row_ids == rid])
            for gid in np.unique(group_ids):
                if gid == rid:
                    assert members == set(t[group_ids == gid])
    # TMEM: four groups x 128 columns = the SM's 512
    assert (threads // 128) * 128 == 512


def stream_row_perm(q, perm_t, perm_g, Q):
    j, r = q & (perm_t - 1), q // perm_t
    return (j // perm_g) * perm_g * (Q // perm_t) + r * perm_g + (j & (perm_g - 1))


def test_streaming_column_kernel_layout(lib):
    v = layout(lib, 4096, 2)
    (n, W, S, threads, warps, groups, G, seg_rows, seg_elems, boxr, seg_bytes, xe, ring_off,
     b_off, bar_off, slot_off, smem) = v[:17]
    xseg = v[17:17 + warps]
    assert (n, W) == (4096, 4) and threads == (n // 64) * W and warps * 32 == threads
    assert groups * 128 == threads and groups * 256 <= 512  # TMEM: 256 columns per group
    assert G == 32 // W and warps * G == n // 64 and seg_rows == G * 64
    assert seg_elems == seg_rows * W and seg_bytes == seg_elems * 8
    assert seg_rows % boxr == 0 and boxr * W * 2 * 4 % 16 == 0  # TMA boxes: whole rows of 32 bytes
    # warps w >= S land in their own span of the exchange: inside it, and
    # disjoint from each other; warps < S use ring slots after the exchange
    for w in range(S, warps):
        assert xseg[w] + seg_elems <= xe
        if w + 1 < warps:
            assert xseg[w] + seg_elems <= xseg[w + 1]
    assert ring_off >= xe * 8 and ring_off % 128 == 0
    assert ring_off + S * seg_bytes <= b_off and b_off % 1024 == 0
    assert bar_off == b_off + 2 * 8192 and slot_off == bar_off + 8 * (warps + 2 * groups)
    assert slot_off + 16 <= smem <= SMEM_MAX
    # stage 0: warp w's butterflies j = w*G .. w*G + G - 1, legs r < 64, read
    # segment element (r*G + j - w*G)*W + c: the segment's rows are block
    # rows w*seg_rows .. + seg_rows, which the row pass fills with column
    # elements j + 64 r in the permuted order
    perm = np.array([stream_row_perm(q, 64, G, n) for q in range(n)])
    assert np.array_equal(np.sort(perm), np.arange(n))
    for w in range(warps):
        j = np.arange(w * G, (w + 1) * G)
        elems = (j[None, :] + 64 * np.arange(64)[:, None]).ravel()
        rows = np.sort(perm[elems])
        assert np.array_equal(rows, np.arange(w * seg_rows, (w + 1) * seg_rows))
        # and the warp reads local row r*G + (j - w*G) for element j + 64 r
        local = perm[j[None, :] + 64 * np.arange(64)[:, None]] - w * seg_rows
        expect = np.arange(64)[:, None] * G + (j - w * G)[None, :]
        assert np.array_equal(local, expect)
    # TMEM columns of a group (base 256 g): D of halves a, b at [0, 64) and
    # [64, 128), A_hi / A_lo of half h at 128 + 64 h + [0, 32) / + [32, 64);
    # MMA block e of half h writes D columns 64 h + 32 e + [0, 32)
    used = np.zeros(256, bool)
    for h in range(2):
        for e in range(2):
            cols = 64 * h + 32 * e + np.arange(32)
            assert not used[cols].any()
            used[cols] = True
        for part in range(2):
            cols = 128 + 64 * h + 32 * part + np.arange(32)
            assert not used[cols].any()
            used[cols] = True
    assert used.all()


@pytest.mark.parametrize("ny,P", [(8192, 2), (4096, 1), (4096, 2)])
def test_permuted_row_store_is_a_bijection(ny, P):
    """The landed row kernels store output q of column block kp at block row
    perm(q) (perm_t = 64, perm_g = 8), i.e. slice row P*perm(q) + kp: every
    slice row is written exactly once."""
    Q = ny // P
    rows = np.array([P * stream_row_perm(q, 64, 8, Q) + kp for kp in range(P) for q in range(Q)])
    assert np.array_equal(np.sort(rows), np.arange(ny))


def test_layout_call_rejects_what_is_not_compiled(lib):
    a = (ctypes.c_longlong * 32)()
    assert lib.fft_debug_tc_layout(512, 0, a) != 0
    assert lib.fft_debug_tc_layout(8192, 2, a) != 0
    assert lib.fft_debug_tc_layout(4096, 3, a) != 0
