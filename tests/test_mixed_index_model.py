"""CPU model of the mixed-radix kernel's index arithmetic (no GPU).

The schedules come from the library (fft_debug_mixed_plan, host only). The
model redoes the kernel's addressing in numpy:
- The stage twiddle tables are laid out in 16-byte pairs. Pair p of
  butterfly k sits at pair index p Ns + k and holds w_{Ns R}^{k r} for
  r = 2p + 1 and 2p + 2. The stage reads pair (r - 1) / 2 for twiddles r,
  r + 1, and every (k, r < R) is written exactly once.
- The four-step row pass's last stage takes lanes transform first
  (c = idx mod W, j = idx / W). It stores output o = j + r Ns of row
  k1 + c at k1 + c + n1 o. Every output position of every transform is
  written exactly once, and a warp's lanes write runs of W adjacent
  positions.
- The L2 prefetch of a CTA's input covers only its own elements: the
  16-byte-aligned interior of its contiguous rows, or one element per row of
  its column group.
"""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2506_15437_gb300 import build
    build.build()
    from paper_2506_15437_gb300 import _native as N
    return N.load()


def schedule(lib, n):
    buf = (ctypes.c_int * 16)()
    n1, n2 = ctypes.c_int(), ctypes.c_int()
    k = lib.fft_debug_mixed_plan(n, buf, ctypes.byref(n1), ctypes.byref(n2))
    return [buf[i] for i in range(k)] if k > 0 else [], (n1.value, n2.value)


def tw_stride(R):
    return (R - 1 + 1) & ~1


@pytest.mark.parametrize("n", [1000, 3000, 4095, 1001, 96, 1728, 2197, 14336, 7])
def test_pair_planar_twiddle_table(lib, n):
    rad, _ = schedule(lib, n)
    assert rad and int(np.prod(rad)) == n
    Ns = 1
    for R in rad:
        M = tw_stride(R)
        count = Ns * M  # float2 entries of the stage's table
        # table kernel: entry e -> pair q = e / 2, p = q / Ns, k = q % Ns, r = 2p + 1 + e % 2
        e = np.arange(count)
        q = e >> 1
        p, k = q // Ns, q % Ns
        r = 2 * p + 1 + (e & 1)
        assert p.max() < M // 2 and k.max() < Ns
        real = r < R
        pairs = set(zip(k[real].tolist(), r[real].tolist()))
        assert len(pairs) == real.sum() == Ns * (R - 1)  # each (k, r) once
        # stage: twiddles r, r + 1 of butterfly k from float4 index ((r - 1) / 2) Ns + k,
        # i.e. float2 entries 2 * that and 2 * that + 1
        for kk in range(0, Ns, max(1, Ns // 7)):
            for rr in range(1, R, 2):
                f4 = ((rr - 1) // 2) * Ns + kk
                assert 2 * f4 + 1 < count
                assert (k[2 * f4], r[2 * f4]) == (kk, rr)
                assert (k[2 * f4 + 1], r[2 * f4 + 1]) == (kk, rr + 1)
        Ns *= R


@pytest.mark.parametrize("n,W", [(10 ** 6, 4), (15360, 8), (6 ** 9, 4), (13 ** 5, 1)])
def test_fourstep_last_stage_stores_once(lib, n, W):
    _, (n1, n2) = schedule(lib, n)
    assert n1 * n2 == n and n1 % W == 0
    rad, _ = schedule(lib, n2)
    R = rad[-1]
    Ns = n2 // R  # the last stage's span: butterflies per row = Ns, k = j
    written = np.zeros(n, dtype=np.int32)
    idx = np.arange(W * Ns)
    c, j = idx % W, idx // W
    for k1 in range(0, n1, W):
        for rr in range(R):
            o = j + rr * Ns
            addr = k1 + c + n1 * o
            written[addr] += 1
            # lanes 0..31 of a warp: runs of W adjacent addresses
            lane = addr[:32].reshape(-1, W)
            assert np.all(np.diff(lane, axis=1) == 1)
    assert written.min() == 1 and written.max() == 1


@pytest.mark.parametrize("n,W,ntrans", [(1000, 4, 8 * 4 - 1), (4095, 1, 5), (1001, 2, 9), (3000, 1, 3)])
def test_row_prefetch_stays_inside_the_group(n, W, ntrans):
    base = 0x1000  # a 16-byte-aligned array start
    for blk in range((ntrans + W - 1) // W):
        t0 = blk * W
        nv = min(W, ntrans - t0)
        a0 = base + t0 * n * 8
        a1 = a0 + nv * n * 8
        p0, p1 = (a0 + 15) & ~15, a1 & ~15
        if p1 > p0:
            assert p0 % 16 == 0 and (p1 - p0) % 16 == 0
            assert a0 <= p0 and p1 <= a1  # only this group's own rows
