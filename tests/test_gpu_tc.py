"""Split-FP16 tensor-core form against the FP64 oracle.

Bar: relative L2 error per transform <= 1e-6 * log2(N) (the FP32 path's is
2e-7 * log2(N)); each test reports both paths' errors on the same input."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, rel_l2, tol_fp32, tol_split_tc, worst_rel_l2

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


@pytest.fixture(params=["tcgen05", "tcgen05_r16", "sync"])
def mma(request, monkeypatch):
    """Which tensor-core butterfly the split plans use: tcgen05 (TMEM
    accumulators; radix-32 stages for lengths 1024..8192, the default),
    tcgen05 held to radix-16 stages, or mma.sync (radix 16)."""
    monkeypatch.setenv("GB300FFT_TC_MMA", "sync" if request.param == "sync" else "tcgen05")
    monkeypatch.setenv("GB300FFT_TC_RADIX", "16" if request.param != "tcgen05" else "32")
    return request.param


def both(g, x, inverse=False):
    ny, nx = x.shape[-2], x.shape[-1]
    batch = x.size // (nx * ny)
    d = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = {}
    for prec in ("split_tc", "fp32"):
        plan = g.Plan(nx, ny, batch, inverse=inverse, precision=prec)
        out[prec] = plan.execute(d).cpu().numpy()
        assert plan.status() == 0
        plan.close()
    return out["split_tc"], out["fp32"]


SHAPES = [(32, 64), (64, 32), (128, 128), (256, 16), (16, 256), (512, 512), (1024, 256),
          (256, 1024), (2048, 64), (64, 2048), (4096, 16), (16, 4096), (8192, 16)]


@pytest.mark.parametrize("ny,nx", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
@pytest.mark.parametrize("inverse", [False, True])
def test_split_tc_small_shapes(g, mma, ny, nx, inverse):
    x = synth.uniform_complex((2, ny, nx), seed=ny * 3 + nx)
    tc, fp = both(g, x, inverse)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    N = nx * ny
    e_tc, e_fp = worst_rel_l2(tc, ref, N), worst_rel_l2(fp, ref, N)
    print(f"split-TC[{mma}] {ny}x{nx} inv={inverse}: rel L2 {e_tc:.3e} (FP32 {e_fp:.3e})")
    assert e_tc <= tol_split_tc(N)
    assert e_fp <= tol_fp32(N)


_REF = {}


def cached_ref(key, fn):
    """Oracle results shared by the two tensor-core butterfly forms."""
    if key not in _REF:
        _REF[key] = fn()
    return _REF[key]


def test_split_tc_8192_exponential_mix(g, mma):
    """U[-1,1) noise + 8 unit exponentials, 8192^2: every output element of
    both paths against the oracle's full transform."""
    n = 8192
    x, freqs = synth.exp_mix_2d(n, n, seed=2506)
    tc, fp = both(g, x)
    ref = cached_ref("8192", lambda: oracle.fft2d(x, threads=ORACLE_THREADS))
    e_tc, e_fp = rel_l2(tc, ref), rel_l2(fp, ref)
    print(f"split-TC[{mma}] 8192^2 exp-mix: whole-output rel L2 {e_tc:.3e} (FP32 {e_fp:.3e})")
    assert e_tc <= tol_split_tc(n * n)
    assert e_fp <= tol_fp32(n * n)
    # the spikes: each exponential puts N = n*n at its bin
    for fy, fx in freqs:
        assert abs(tc[fy, fx] - n * n) / (n * n) < 1e-3


def test_split_tc_1d_batch_4096(g, mma):
    """16384 signals of length 4096 (noise + 8 exponentials per signal):
    every signal of both paths against the oracle."""
    x, _ = synth.exp_mix_1d(16384, 4096, seed=2506)
    d = torch.from_numpy(x).cuda()
    plan = g.Plan(4096, 1, 16384, precision="split_tc")
    tc = plan.execute(d).cpu().numpy()
    assert plan.status() == 0
    plan.close()
    fp = g.get_plan(4096, 1, 16384, False, "fp32", "cuda").execute(d).cpu().numpy()
    ref = cached_ref("1d4096", lambda: oracle.fft1d_batch(x, threads=ORACLE_THREADS))
    e_tc, e_fp = worst_rel_l2(tc, ref, 4096), worst_rel_l2(fp, ref, 4096)
    print(f"split-TC[{mma}] 1D 4096 x 16384: worst per-signal rel L2 {e_tc:.3e} (FP32 {e_fp:.3e})")
    assert e_tc <= tol_split_tc(4096)
    assert e_fp <= tol_fp32(4096)


def test_split_tc_handles_large_dynamic_range(g, mma):
    """Per-butterfly power-of-two scaling: inputs spanning 1e-20..1e20 stay
    accurate (no float16 overflow or flush)."""
    n = 256
    x = synth.uniform_complex((n, n), seed=4).astype(np.complex128)
    x *= np.logspace(-20, 20, n)[:, None]
    x = x.astype(np.complex64)
    tc, _ = both(g, x)
    ref = oracle.fft2d(x, threads=ORACLE_THREADS)
    assert np.isfinite(tc).all()
    assert rel_l2(tc, ref) <= tol_split_tc(n * n)


def test_split_tc_unsupported_shapes_fail_loudly(g):
    from paper_2506_15437_gb300 import FFTError
    with pytest.raises(FFTError):
        g.Plan(8, 8, 1, precision="split_tc")   # no radix-16 stage at all
    with pytest.raises(FFTError):
        g.Plan(16, 16, 1, precision="split_tc")  # a 16-row column tile needs 32 columns for a full warp


def test_split_tc_default_is_tcgen05(g):
    plan = g.Plan(256, 256, 1, precision="split_tc")
    d = plan.describe()
    assert d["rows"]["kernel"].startswith("k_rows_tcgen05")
    assert d["cols"]["kernel"].startswith("k_cols_tcgen05")
    # lengths 1024..8192: radix-32 tensor-core stages
    plan = g.Plan(8192, 8192, 1, precision="split_tc")
    d = plan.describe()
    assert d["rows"]["kernel"].startswith("k_rows_tc32_land") and d["rows"]["radices"] == [8, 32, 32]
    # the rows pre-split the columns by 2: 4096-point column blocks, streamed
    # as two radix-64 stages (each a radix-2 level and two radix-32 products)
    assert d["split"] == 2
    assert d["cols"]["kernel"].startswith("k_cols_tc_stream") and d["cols"]["radices"] == [64, 64]
    plan.close()


@pytest.mark.parametrize("ny,nx,batch", [(1024, 1024, 1), (2048, 2048, 1), (4096, 4096, 1), (1024, 16, 3),
                                         (2048, 16, 2), (4096, 16, 2), (8192, 16, 1), (32, 8192, 2),
                                         (8192, 64, 1), (16, 1024, 5), (8192, 1024, 1), (4096, 2048, 2),
                                         (1, 1024, 7), (1, 8192, 3), (1, 4096, 3), (1, 2048, 40)])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("form", ["land", "tmem", "smem"])
def test_radix32_tensor_core_shapes(g, monkeypatch, ny, nx, batch, inverse, form):
    """Radix-32 tcgen05 stages on every compiled row length and column tile
    (rows of 1024..8192 points; columns of 1024, 2048, 4096, 8192 points in
    16-, 8-, 4- and 2-column tiles; the column pre-split at ny = 8192), both
    directions, against the oracle.  Forms: rows from landed units (where the
    rows divide into whole units; the rest fall back), A in tensor memory, A
    in shared memory."""
    monkeypatch.setenv("GB300FFT_TC_MMA", "tcgen05")
    monkeypatch.setenv("GB300FFT_TC_RADIX", "32")
    monkeypatch.setenv("GB300FFT_TC_TMEM_A", "0" if form == "smem" else "1")
    monkeypatch.setenv("GB300FFT_TC_LAND", "1" if form == "land" else "0")
    tmem_a = "0" if form == "smem" else "1"
    plan = g.Plan(nx, ny, batch, inverse=inverse, precision="split_tc")
    d = plan.describe()
    x = synth.uniform_complex((batch, ny, nx), seed=7 * ny + nx + batch)
    got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    plan.close()
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    N = nx * ny
    err = worst_rel_l2(got, ref, N)
    print(f"tc32 A@{'tmem' if tmem_a == '1' else 'smem'} {ny}x{nx}x{batch} inv={inverse} rows={d['rows']['kernel']} "
          f"cols={d['cols']['kernel']}: {err:.3e}")
    assert err <= tol_split_tc(N)
    land = False
    if nx >= 1024:
        assert d["rows"]["kernel"].startswith("k_rows_tc32")
        nrows = ny * batch
        units = 512 // (nx // 32)  # rows per landed unit of the pre-split form
        rs = max(1, 128 // (nx // 32))  # rows per sub-unit of the unsplit form
        land = form == "land" and (nrows % rs == 0 if d["split"] == 1 else (ny // 2) % (units // 2) == 0)
        assert d["rows"]["kernel"].startswith("k_rows_tc32_land") == land
    if ny >= 1024 and nx > 1:
        stream = land and d["cols"]["n"] == 4096 and nx % 4 == 0
        assert d["cols"]["kernel"].startswith("k_cols_tc_stream" if stream else "k_cols_tc32")


@pytest.mark.parametrize("ny,nx,batch", [(8192, 8192, 1), (4096, 1024, 2), (8192, 1024, 2), (4096, 4096, 1),
                                         (8192, 2048, 1)])
@pytest.mark.parametrize("inverse", [False, True])
def test_streaming_tensor_core_columns(g, monkeypatch, ny, nx, batch, inverse):
    """Streaming split-FP16 column pass (4096-point blocks, two radix-64
    stages of a float32 radix-2 level and two radix-32 tensor-core products,
    rows stored permuted by the landed row pass): out of place against the
    oracle, element by element over every slice; in place (unsplit, no
    permutation, the radix-32 column pass) too; the result agrees with the
    non-streaming pass within the bound."""
    monkeypatch.setenv("GB300FFT_TC_MMA", "tcgen05")
    monkeypatch.setenv("GB300FFT_TC_RADIX", "32")
    plan = g.Plan(nx, ny, batch, inverse=inverse, precision="split_tc")
    monkeypatch.setenv("GB300FFT_TC_STREAM", "0")
    plain = g.Plan(nx, ny, batch, inverse=inverse, precision="split_tc")
    monkeypatch.delenv("GB300FFT_TC_STREAM")
    d = plan.describe()
    assert d["cols"]["kernel"].startswith("k_cols_tc_stream") and d["cols"]["radices"] == [64, 64]
    assert plain.describe()["cols"]["kernel"].startswith("k_cols_tc32")
    x = synth.uniform_complex((batch, ny, nx), seed=5 * ny + nx + batch)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    xd = torch.from_numpy(x).cuda()
    got = plan.execute(xd).cpu().numpy()
    assert plan.status() == 0
    N = nx * ny
    err = worst_rel_l2(got, ref, N)
    print(f"tc stream {ny}x{nx}x{batch} inv={inverse}: {err:.3e}")
    assert err <= tol_split_tc(N)
    other = plain.execute(xd).cpu().numpy()
    assert worst_rel_l2(other, ref, N) <= tol_split_tc(N)
    plan.execute(xd, out=xd)  # in place: no permuted intermediate
    assert plan.status() == 0
    assert worst_rel_l2(xd.cpu().numpy(), ref, N) <= tol_split_tc(N)
    plan.close()
    plain.close()


@pytest.mark.parametrize("ny,nx,split", [(8192, 1024, "2"), (8192, 1024, "1"), (4096, 4096, "2"), (4096, 1024, "1")])
def test_radix32_column_presplit_choices(g, monkeypatch, ny, nx, split):
    """The radix-32 row pass pre-splits the columns by 1 or 2 (the 2-point
    DFT across rows q and q + ny/2 and the twiddle w_ny^q); every choice gives
    the transform within the bound, out of place and in place (in place runs
    unsplit)."""
    monkeypatch.setenv("GB300FFT_TC_MMA", "tcgen05")
    monkeypatch.setenv("GB300FFT_TC_RADIX", "32")
    monkeypatch.setenv("GB300FFT_TC_SPLIT", split)
    plan = g.Plan(nx, ny, 1, precision="split_tc")
    monkeypatch.delenv("GB300FFT_TC_SPLIT")
    d = plan.describe()
    assert d["split"] == int(split)
    assert d["cols"]["n"] == ny // int(split)
    x = synth.uniform_complex((ny, nx), seed=ny + nx + int(split))
    ref = oracle.fft2d(x, threads=ORACLE_THREADS)
    xd = torch.from_numpy(x).cuda()
    got = plan.execute(xd).cpu().numpy()
    assert plan.status() == 0
    assert rel_l2(got, ref) <= tol_split_tc(nx * ny)
    plan.execute(xd, out=xd)
    assert plan.status() == 0
    assert rel_l2(xd.cpu().numpy(), ref) <= tol_split_tc(nx * ny)
    plan.close()
