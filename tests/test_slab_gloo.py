"""Slab-decomposed 2D transform over gloo ranks on the CPU (no GPU).

SlabFFT2 (paper_2506_15437_gb300/slab.py) is the multi-GPU driver: local row
FFTs, pack, one all-to-all, unpack, local column FFTs.  Here it runs over
world_size 2 and 4 gloo process groups with CPU stand-ins for the local steps
-- the FP64 oracle for the row and column FFTs and numpy restatements of the
pack / unpack index maps the library's kernels implement (the GPU tests check
those kernels against the same maps) -- so the decomposition, the chunk
layout and the exchange are checked exactly: every rank's column slab equals
the matching columns of the oracle's whole 2D transform.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def pack_ref(y, parts, batch, rows, nx):
    """out[s][b][y][x'] = y[b][y][s*w + x']"""
    w = nx // parts
    return np.ascontiguousarray(y.reshape(batch, rows, parts, w).transpose(2, 0, 1, 3))


def unpack_ref(recv, parts, batch, rows, w):
    """out[b][r*rows + y][x'] = recv[r][b][y][x']"""
    return np.ascontiguousarray(recv.reshape(parts, batch, rows, w).transpose(1, 0, 2, 3).reshape(batch, parts * rows, w))


class CpuOps:
    """The slab driver's local steps on the CPU: FP64 oracle transforms and
    the numpy index maps (complex128 torch tensors in and out)."""

    def __init__(self, inverse):
        self.dir = 1 if inverse else -1

    def rows_fft(self, x):
        import oracle
        return torch.from_numpy(oracle.fft1d_any(x.numpy(), dir=self.dir))

    def pack(self, y, parts, batch, rows, nx):
        return torch.from_numpy(pack_ref(y.numpy(), parts, batch, rows, nx))

    def unpack(self, recv, parts, batch, rows, w):
        return torch.from_numpy(unpack_ref(recv.numpy(), parts, batch, rows, w))

    def cols_fft(self, z):
        import oracle
        zt = np.ascontiguousarray(z.numpy().transpose(0, 2, 1))  # [b][w][ny]
        return torch.from_numpy(np.ascontiguousarray(oracle.fft1d_any(zt, dir=self.dir).transpose(0, 2, 1)))

    def empty_like(self, t):
        return torch.empty_like(t)


def _rank(rank, world, port, cases, queue):
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2506_15437_gb300.slab import SlabFFT2
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for case, (nx, ny, batch, inverse) in enumerate(cases):
            x = synth.uniform_complex((batch, ny, nx), seed=ny + nx + world).astype(np.complex128)
            rows, w = ny // world, nx // world
            mine = np.ascontiguousarray(x[:, rank * rows:(rank + 1) * rows, :])
            slab = SlabFFT2(nx, ny, batch, inverse=inverse, ops=CpuOps(inverse))
            got = slab(torch.from_numpy(mine)).numpy()
            ref = oracle.fft2d_any(x, dir=1 if inverse else -1)[:, :, rank * w:(rank + 1) * w]
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            queue.put((case, rank, got.shape, err))
    finally:
        dist.destroy_process_group()


# (nx, ny, batch, inverse): powers of two, a batch of slices, both directions,
# and a width that leaves 3 columns per rank
CASES = {2: [(64, 32, 1, False), (32, 64, 3, True), (6, 4, 2, False)],
         4: [(128, 64, 2, False), (64, 128, 1, True), (12, 8, 1, True)]}


@pytest.mark.parametrize("world", [2, 4])
def test_slab_fft_over_gloo_matches_the_oracle(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    cases = CASES[world]
    port = 29611 + 17 * world
    procs = [ctx.Process(target=_rank, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=180) for _ in range(world * len(cases))]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for case, (nx, ny, batch, _) in enumerate(cases):
        got = [(rank, shape, err) for c, rank, shape, err in results if c == case]
        assert sorted(r for r, _, _ in got) == list(range(world))
        for rank, shape, err in got:
            assert shape == (batch, ny, nx // world)
            assert err < 1e-12, (case, rank, err)


def test_pack_unpack_maps_invert_the_slab_layout():
    """unpack(exchange(pack(...))) over all ranks rebuilds each rank's
    column slab of the full array: the index maps, checked alone."""
    rng = np.random.default_rng(5)
    G, batch, ny, nx = 4, 2, 16, 12
    rows, w = ny // G, nx // G
    full = rng.standard_normal((batch, ny, nx)) + 1j * rng.standard_normal((batch, ny, nx))
    sends = [pack_ref(np.ascontiguousarray(full[:, r * rows:(r + 1) * rows]), G, batch, rows, nx) for r in range(G)]
    for s in range(G):
        recv = np.stack([sends[r][s] for r in range(G)])  # what rank s receives, by source rank
        assert np.array_equal(unpack_ref(recv, G, batch, rows, w), full[:, :, s * w:(s + 1) * w])
