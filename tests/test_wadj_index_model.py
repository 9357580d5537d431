"""CPU model of the fused differentiation form's column pass (no GPU).

`k_cols_wadj<N, E, W>` works on tiles of W adjacent columns of one [N][nx]
slice; tile `id` is column group id % (nx / W) of slice id / (nx / W).  Per
tile it:
- lands the tile by TMA boxes of BOXR rows from a map over y, coordinates
  (x = 2 W gx floats, 0, slice N + k BOXR);
- sweeps the tile in natural order, element k = i W + c reading the weight
  at i nx + c of the slice;
- stores the adjoint's column half at i nx + c;
- writes one partial per tile at partials[id].
The model redoes that address arithmetic with numpy and checks three
properties. Every box lies inside the map, starting on a 16-byte boundary.
The sweep and the stores each touch every element of the array exactly
once, with offsets inside a slice that fit 32 bits. There is one partial
per tile.
It also checks the plan's tile-width rule for the fused form: the default
widest tile of at most 64 KiB, covered only when a CTA is whole warps.
"""
import numpy as np
import pytest


def default_col_w(n, nx):
    # the column pass's default width: 64 KiB tiles below 4096 points
    w = (16384 if n >= 4096 else 8192) // n
    w = max(2, min(16, w))
    while w > nx:
        w >>= 1
    return w


def fused_width(n, nx):
    """W of the fused pass, or 0 where the plan reports no fused form."""
    if n > 2048 or n < 32 or n & (n - 1):
        return 0
    w = default_col_w(n, nx)
    while w > 2 and n * w * 8 > 65536:
        w >>= 1
    threads = (n // 16) * w  # E = 16 below 4096 points
    return w if nx % w == 0 and threads % 32 == 0 else 0


@pytest.mark.parametrize("n,nx,batch", [(64, 64, 1), (256, 1024, 3), (1024, 256, 2), (2048, 2048, 2),
                                        (32, 4096, 1), (2048, 64, 2)])
def test_fused_column_pass_touches_every_element_once(n, nx, batch):
    W = fused_width(n, nx)
    assert W > 0
    assert n * W * 8 <= 65536
    boxr = min(n, 256)
    groups_x = nx // W
    ntiles = groups_x * batch
    map_dims = (2 * nx, 1, n * batch)
    swept = np.zeros(n * nx * batch, dtype=np.int32)
    stored = np.zeros_like(swept)
    parts = np.zeros(ntiles, dtype=np.int32)
    i = np.arange(n)[:, None]
    c = np.arange(W)[None, :]
    for tid in range(ntiles):
        b, gx = divmod(tid, groups_x)
        off = b * n * nx + gx * W
        # TMA boxes
        x = gx * 2 * W
        assert (x * 4) % 16 == 0
        for k in range(n // boxr):
            z = b * n + k * boxr
            assert 0 <= x and x + 2 * W <= map_dims[0]
            assert 0 <= z and z + boxr <= map_dims[2]
        # the sweep: element k = i W + c of the tile, weight at i nx + c
        k = (i * W + c).ravel()
        assert np.array_equal(np.sort(k), np.arange(n * W))
        rel = (k // W) * nx + (k % W)
        assert rel.max() < 2 ** 31 and rel.max() < n * nx
        swept[off + rel] += 1
        # the stores of the adjoint's column half: output i of column c
        stored[(off + i * nx + c).ravel()] += 1
        parts[tid] += 1
    assert swept.min() == 1 and swept.max() == 1
    assert stored.min() == 1 and stored.max() == 1
    assert parts.min() == 1 and parts.max() == 1


def test_fused_width_rule():
    """Whole warps only; 64 KiB tiles at most; columns up to 2048 points."""
    for n in [2 ** k for k in range(1, 14)]:
        for nx in [2 ** k for k in range(1, 14)]:
            W = fused_width(n, nx)
            if W == 0:
                continue
            assert 32 <= n <= 2048 and W <= nx and nx % W == 0
            assert ((n // 16) * W) % 32 == 0 and n * W * 8 <= 65536
    # the bench's and the tests' shapes are covered
    assert fused_width(2048, 2048) == 4 and fused_width(1024, 1024) == 8 and fused_width(64, 64) == 16
    # columns of 4096 points and more are not
    assert fused_width(4096, 4096) == 0 and fused_width(8192, 16) == 0
