"""CPU model of the streaming column pass's TMA output stores (no GPU).

The column pass transforms tiles of W = 4 adjacent columns of a length-4096
column block (rows kp + P*ky of slice b, ky < 4096) with T = 64 butterflies
per column and E = 64 outputs per thread: thread (tt, c) ends with output
rows ky = tt + T*k, k < E, of column c.  With TMA stores each warp (G = 8
adjacent butterflies tt) stages KB = 8 consecutive k at a time as a box of
the 4D map {floats of a row, kp, ky mod T, slice*E + ky / T} and stores it.
The model checks that every box lies inside the map, that every staged
value lands exactly where the plain store would put it, and that a launch
writes every output element exactly once (Section 5's column FFTs write
natural order, in place on the rows they read).
"""
import numpy as np
import pytest

N, E, W, KB = 4096, 64, 4, 8
T = N // E
G = 32 // W
WARPS = T * W // 32


def plain_address(nx, P, b, kp, gx, ky, c):
    return (b * N * P + kp + P * ky) * nx + gx * W + c


@pytest.mark.parametrize("nx,P,batch", [(4, 1, 1), (64, 2, 1), (8, 2, 3), (8192, 2, 1), (4096, 1, 2)])
def test_tma_store_boxes_cover_the_output_once(nx, P, batch):
    rows = N * P * batch  # ny * batch with ny = P * N
    dims = (2 * nx, P, T, rows // (P * T))
    groups_x = nx // W
    written = np.zeros(rows * nx, dtype=np.int32)
    kk = np.arange(KB)[:, None, None]
    ttl = np.arange(G)[None, :, None]
    c = np.arange(W)[None, None, :]
    for tile in range(groups_x * P * batch):
        blk, gx = divmod(tile, groups_x)
        b, kp = divmod(blk, P)
        xo = gx * 2 * W
        kb0 = b * E
        for warp in range(WARPS):
            for rr in range(E // KB):
                box0 = (xo, kp, warp * G, kb0 + rr * KB)
                box = (2 * W, 1, G, KB)
                for d in range(4):
                    assert 0 <= box0[d] and box0[d] + box[d] <= dims[d], (d, box0, dims)
                assert (box0[0] * 4) % 16 == 0  # innermost coordinate on a 16-byte boundary
                # staged element (kk, ttl, c) sits at box position (2c, 0, ttl, kk)
                g_row = box0[1] + P * ((box0[3] + kk) * T + (box0[2] + ttl))  # row index kp + P*r
                addr = g_row * nx + (box0[0] // 2 + c)
                # the value there is output k = rr*KB + kk of thread tt = warp*G + ttl, column c
                ky = (warp * G + ttl) + T * (rr * KB + kk)
                want = plain_address(nx, P, b, kp, gx, ky, c)
                assert np.array_equal(np.broadcast_to(addr, want.shape), want)
                written[addr.ravel()] += 1
    assert written.min() == 1 and written.max() == 1


def test_staging_chunks_fit_the_shared_memory_budget():
    pad = lambda f: f + (f >> 6)  # noqa: E731  (E = 64 exchange padding)
    xch = (pad(N * W - 1) + 1) * 8
    ring_off = (xch + 127) // 128 * 128
    ring = 4 * (G * E * W * 8)
    staging = WARPS * 2 * KB * G * W * 8
    total = ring_off + ring + staging + 8 * WARPS + 16
    assert (KB * G * W * 8) % 128 == 0  # each chunk starts 128-byte aligned
    assert total + 128 <= 232448  # dynamic + static shared memory of one CTA
