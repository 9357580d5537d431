"""The library's pieces of the slab-decomposed 2D transform on one GPU.

* fft_slab_pack / fft_slab_unpack against numpy restatements of their index
  maps, bit for bit (both the 16-byte and the 8-byte element paths).
* The column-only plan against the oracle's column transforms, both
  directions, out of place and in place.
* The whole slab algorithm for G = 2, 4, 8 ranks emulated on one GPU: each
  virtual rank runs its row plan and the pack kernel, the all-to-all is plain
  device copies between the ranks' buffers (no kernel of one rank waits on
  another's), then each rank unpacks and runs its column plan; the column
  slabs together are compared whole with the oracle.  The exchange itself
  runs over gloo ranks in tests/test_slab_gloo.py.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, rel_l2, tol_fp32
from tests.test_slab_gloo import pack_ref, unpack_ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_15437_gb300 import build
    build.build()
    import paper_2506_15437_gb300 as g
    return g


@pytest.mark.parametrize("parts,batch,rows,nx", [(2, 1, 8, 64), (4, 3, 5, 32), (8, 2, 16, 8192), (3, 2, 7, 9),
                                                 (4, 1, 2, 12)])
def test_pack_unpack_kernels_match_the_index_maps(g, parts, batch, rows, nx):
    x = synth.uniform_complex((batch, rows, nx), seed=parts * 100 + rows)
    got = g.slab_pack(torch.from_numpy(x).cuda(), parts, batch, rows, nx).cpu().numpy()
    assert np.array_equal(got, pack_ref(x, parts, batch, rows, nx))
    w = nx // parts
    r = synth.uniform_complex((parts, batch, rows, w), seed=parts * 7 + w)
    got = g.slab_unpack(torch.from_numpy(r).cuda(), parts, batch, rows, w).cpu().numpy()
    assert np.array_equal(got, unpack_ref(r, parts, batch, rows, w))


@pytest.mark.parametrize("ny,nx,batch", [(8192, 16, 1), (4096, 1024, 1), (1024, 2, 3), (2, 64, 2), (512, 4096, 2)])
@pytest.mark.parametrize("inverse", [False, True])
def test_column_plan_against_the_oracle(g, ny, nx, batch, inverse):
    x = synth.uniform_complex((batch, ny, nx), seed=ny + nx)
    d = 1 if inverse else -1
    xt = np.ascontiguousarray(x.transpose(0, 2, 1))
    ref = np.ascontiguousarray(oracle.fft1d_batch(xt, dir=d, threads=ORACLE_THREADS).transpose(0, 2, 1))
    plan = g.ColumnPlan(nx, ny, batch, inverse=inverse)
    assert plan.describe()["rows"]["kernel"] == "none"
    xd = torch.from_numpy(x).cuda()
    got = plan.execute(xd).cpu().numpy()
    assert plan.status() == 0
    for b in range(batch):
        assert rel_l2(got[b], ref[b]) <= tol_fp32(ny)
    plan.execute(xd, out=xd)  # in place
    assert rel_l2(xd.cpu().numpy(), ref) <= tol_fp32(ny)
    plan.close()


def test_column_plan_rejects_what_it_does_not_cover(g):
    from paper_2506_15437_gb300 import _native as N
    lib = N.load()
    assert lib.fft_plan_create_columns(64, 16384, 1, -1, 0) is None  # columns beyond 8192
    assert lib.fft_last_error() == N.FFT_ERR_INVALID_SIZE
    assert lib.fft_plan_create_columns(64, 64, 1, -1, 1) is None  # split-FP16 form
    assert lib.fft_last_error() == N.FFT_ERR_UNSUPPORTED
    assert lib.fft_plan_create_columns(48, 64, 1, -1, 0) is None  # not a power of two
    assert lib.fft_last_error() == N.FFT_ERR_INVALID_SIZE


@pytest.mark.parametrize("G,nx,ny,batch,inverse", [(2, 1024, 512, 1, False), (4, 256, 1024, 2, True),
                                                   (8, 8192, 1024, 1, False), (2, 64, 8192, 1, False)])
def test_slab_algorithm_with_virtual_ranks(g, G, nx, ny, batch, inverse):
    from paper_2506_15437_gb300.slab import LibraryOps
    x = synth.uniform_complex((batch, ny, nx), seed=G * 31 + nx)
    rows, w = ny // G, nx // G
    xd = torch.from_numpy(x).cuda()
    ops = [LibraryOps(nx, ny, batch, G, inverse) for _ in range(G)]
    sends = []
    for r in range(G):
        mine = xd[:, r * rows:(r + 1) * rows, :].contiguous()
        y = ops[r].rows_fft(mine)
        sends.append(ops[r].pack(y, G, batch, rows, nx))
    torch.cuda.synchronize()
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    out = np.empty_like(ref)
    for s in range(G):
        recv = torch.stack([sends[r][s] for r in range(G)])  # the exchange, as device copies
        z = ops[s].unpack(recv, G, batch, rows, w)
        out[:, :, s * w:(s + 1) * w] = ops[s].cols_fft(z).cpu().numpy()
    for b in range(batch):
        assert rel_l2(out[b], ref[b]) <= tol_fp32(nx * ny)


def test_slab_driver_on_one_rank(g):
    """SlabFFT2 without a process group: one rank, no exchange, the whole
    transform (row plan, pack, unpack, column plan)."""
    from paper_2506_15437_gb300.slab import SlabFFT2
    nx, ny, batch = 2048, 1024, 2
    x = synth.uniform_complex((batch, ny, nx), seed=3)
    got = SlabFFT2(nx, ny, batch)(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fft2d(x, threads=ORACLE_THREADS)
    for b in range(batch):
        assert rel_l2(got[b], ref[b]) <= tol_fp32(nx * ny)
