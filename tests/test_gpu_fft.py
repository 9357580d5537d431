"""GPU parity of the plain FP32 path against the FP64 oracle (same seeded
inputs on both sides), through the C ABI via the ctypes binding.

Bar: relative L2 error per transform <= 2e-7 * log2(nx*ny); the reorder
index maps bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, digit_reversal, rel_l2, tol_fp32, worst_rel_l2

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


def run_plan(g, x: np.ndarray, inverse=False, inplace=False):
    ny, nx = x.shape[-2], x.shape[-1]
    batch = x.size // (nx * ny)
    plan = g.get_plan(nx, ny, batch, inverse, "fp32", "cuda")
    d = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = plan.execute(d, out=d if inplace else None)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return out.cpu().numpy()


def check_full(g, x, inverse=False, inplace=False):
    ny, nx = x.shape[-2], x.shape[-1]
    got = run_plan(g, x, inverse, inplace)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    err = worst_rel_l2(got, ref, nx * ny)
    assert err <= tol_fp32(nx * ny), (x.shape, inverse, err, tol_fp32(nx * ny))
    return err


# every power-of-two shape with nx*ny <= 2^16 and a ragged batch of 3
SHAPES = [(1 << ly, 1 << lx) for ly in range(0, 14) for lx in range(0, 14)
          if (1 << lx) * (1 << ly) <= (1 << 16)]


@pytest.mark.parametrize("ny,nx", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
def test_small_shapes_forward_and_inverse(g, ny, nx):
    x = synth.uniform_complex((3, ny, nx), seed=1000 + 31 * nx + ny)
    check_full(g, x, inverse=False)
    check_full(g, x, inverse=True)


def test_config1_256x256(g):
    x = synth.uniform_complex((256, 256), seed=2506)
    err = check_full(g, x)
    assert err < 2e-7 * 16


@pytest.mark.parametrize("n", [1024, 2048, 4096])
@pytest.mark.parametrize("inverse", [False, True])
def test_config2_square_full(g, n, inverse):
    x = synth.normal_complex((n, n), seed=2506)
    check_full(g, x, inverse=inverse)


@pytest.mark.parametrize("inverse", [False, True])
def test_config2_8192_full(g, inverse):
    """8192^2 in the bench's launch configuration (landed-pair rows with the
    column pre-split, streaming planar columns): every output element
    against the oracle's full transform of the same input."""
    n = 8192
    x = synth.normal_complex((n, n), seed=2506)
    got = run_plan(g, x, inverse)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    err = rel_l2(got, ref)
    print(f"8192^2 inverse={inverse}: whole-output rel L2 {err:.3e} (bound {tol_fp32(n * n):.2e})")
    assert err <= tol_fp32(n * n)


@pytest.mark.parametrize("ny,nx", [(8192, 2), (2, 8192), (8192, 16), (16, 8192), (4096, 64),
                                   (32, 4096), (8192, 8), (1, 8192), (8192, 1)])
def test_extreme_aspect_ratios(g, ny, nx):
    x = synth.uniform_complex((ny, nx), seed=ny + 7 * nx)
    check_full(g, x)
    check_full(g, x, inverse=True)


def test_batched_2d(g):
    x = synth.uniform_complex((5, 128, 512), seed=3)
    check_full(g, x)


def test_batch_of_1d_signals_4096(g):
    """nx=4096, ny=1, batch 16384 (the 1D batch workload): every signal."""
    x, _ = synth.exp_mix_1d(16384, 4096, seed=2506)
    plan = g.get_plan(4096, 1, 16384, False, "fp32", "cuda")
    out = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fft1d_batch(x, threads=ORACLE_THREADS)
    err = worst_rel_l2(out, ref, 4096)
    print(f"1D 4096 x 16384: worst per-signal rel L2 {err:.3e}")
    assert err <= tol_fp32(4096)


def test_exponential_spikes_2048(g):
    """Unit exponentials land exactly on their bins (N there, ~0 elsewhere)."""
    n = 2048
    x, freqs = synth.exp_mix_2d(n, n, seed=11)
    noise_free = np.zeros((n, n), np.complex64)
    yy = np.arange(n)[:, None]
    xx = np.arange(n)[None, :]
    for fy, fx in freqs:
        noise_free += np.exp(2j * np.pi * (((fx * xx) % n) / n + ((fy * yy) % n) / n)).astype(np.complex64)
    got = run_plan(g, noise_free)
    want = np.zeros((n, n), np.complex128)
    for fy, fx in freqs:
        want[fy, fx] += n * n
    assert rel_l2(got, want) < 2e-7 * 22


def test_inplace_equals_out_of_place(g):
    x = synth.normal_complex((2, 1024, 2048), seed=5)
    a = run_plan(g, x, inplace=False)
    b = run_plan(g, x, inplace=True)
    assert np.array_equal(a, b)


def test_inverse_of_forward_is_N_times_identity(g):
    n = 1024
    x = synth.uniform_complex((n, n), seed=9)
    d = torch.from_numpy(x).cuda()
    X = g.get_plan(n, n, 1, False, "fp32", "cuda").execute(d)
    y = g.get_plan(n, n, 1, True, "fp32", "cuda").execute(X)
    assert rel_l2(y.cpu().numpy(), n * n * x.astype(np.complex128)) <= 2 * tol_fp32(n * n)


def test_adjoint_dot_product(g):
    """<F x, y> == <x, F^H y>: fft_backward is the conjugate transpose."""
    ny, nx = 512, 256
    x = synth.uniform_complex((ny, nx), seed=1)
    y = synth.uniform_complex((ny, nx), seed=2)
    plan = g.get_plan(nx, ny, 1, False, "fp32", "cuda")
    Fx = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
    FHy = plan.backward(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(y.astype(np.complex128), Fx)
    rhs = np.vdot(FHy, x.astype(np.complex128))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_graph_capture_matches_eager(g):
    n = 1024
    x = torch.from_numpy(synth.uniform_complex((n, n), seed=4)).cuda()
    plan = g.get_plan(n, n, 1, False, "fp32", "cuda")
    out = torch.empty_like(x)
    eager = plan.execute(x).clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.execute(x, out=out)  # warm the tensor-map cache outside capture
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.execute(x, out=out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)


def test_misaligned_pointer_rejected(g):
    n = 64
    buf = torch.zeros(n * n + 1, dtype=torch.complex64, device="cuda")
    plan = g.get_plan(n, n, 1, False, "fp32", "cuda")
    from paper_2506_15437_gb300 import _native as N
    lib = N.load()
    rc = lib.fft_execute(plan._p, buf.data_ptr() + 8, buf.data_ptr() + 8,
                         torch.cuda.current_stream().cuda_stream)
    assert rc == N.FFT_ERR_INVALID_ARG


def test_rejects_wrong_dtype_and_size(g):
    plan = g.get_plan(64, 64, 1, False, "fp32", "cuda")
    with pytest.raises(TypeError):
        plan.execute(torch.zeros(64, 64, dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):
        plan.execute(torch.zeros(64, 32, dtype=torch.complex64, device="cuda"))


@pytest.mark.parametrize("axis", [0, 1])
def test_reorder_map_bit_exact(g, axis):
    """The kernels' data movement alone (identity butterflies) is exactly the
    mixed-radix digit reversal of their stage radices, for every length."""
    for L in range(1, 14):
        n = 1 << L
        m = g.reorder_map(n, axis).cpu().numpy().astype(np.int64)
        rad = g.radices(n, axis)
        assert np.array_equal(np.sort(m), np.arange(n)), (n, "not a bijection")
        assert np.array_equal(m, digit_reversal(n, rad)), (n, axis, rad)


@pytest.mark.parametrize("ny,nx,batch", [(16, 8, 3), (64, 32, 2), (256, 128, 1), (1024, 16, 2),
                                         (4096, 4, 1), (8192, 2, 1)])
@pytest.mark.parametrize("inverse", [False, True])
def test_forced_column_presplit(g, monkeypatch, ny, nx, batch, inverse):
    """The column pre-split (2-point DFT across rows y, y + ny/2 in the row
    pass, length-ny/2 columns after) forced on shapes that would not use it."""
    monkeypatch.setenv("GB300FFT_SPLIT", "2")
    plan = g.Plan(nx, ny, batch, inverse=inverse)
    monkeypatch.delenv("GB300FFT_SPLIT")
    x = synth.uniform_complex((batch, ny, nx), seed=ny * nx + batch)
    got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    assert worst_rel_l2(got, ref, nx * ny) <= tol_fp32(nx * ny)
    plan.close()


def test_presplit_inplace_falls_back_to_unsplit(g):
    """In place, the pre-split pairing would overwrite rows a partner CTA
    still reads, so in-place calls take the unsplit path; both agree."""
    ny, nx = 8192, 64
    x = synth.normal_complex((ny, nx), seed=21)
    a = run_plan(g, x, inplace=False)
    b = run_plan(g, x, inplace=True)
    ref = oracle.fft2d(x, threads=ORACLE_THREADS)
    assert rel_l2(a, ref) <= tol_fp32(nx * ny)
    assert rel_l2(b, ref) <= tol_fp32(nx * ny)


@pytest.mark.parametrize("e", ["16", "32"])
@pytest.mark.parametrize("ny,nx,batch,split", [(2048, 8, 2, "1"), (4096, 4, 1, "1"), (4096, 16, 1, "2"),
                                               (8192, 4, 1, "2"), (8192, 2, 1, "1"), (2048, 64, 1, "1")])
@pytest.mark.parametrize("inverse", [False, True])
def test_column_pass_by_cta_pairs(g, monkeypatch, e, ny, nx, batch, split, inverse):
    """Column pass by 2-CTA clusters (radix-2 split of each column block,
    both halves loaded by both CTAs, cluster barrier before the in-place
    stores), forced on; out of place and in place."""
    monkeypatch.setenv("GB300FFT_COL_PAIR", "1")
    monkeypatch.setenv("GB300FFT_COL_E", e)
    monkeypatch.setenv("GB300FFT_SPLIT", split)
    plan = g.Plan(nx, ny, batch, inverse=inverse)
    for k in ("GB300FFT_COL_PAIR", "GB300FFT_COL_E", "GB300FFT_SPLIT"):
        monkeypatch.delenv(k)
    assert plan.describe()["cols"]["kernel"].startswith("k_cols_pair")
    x = synth.uniform_complex((batch, ny, nx), seed=ny + nx + batch)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    d = torch.from_numpy(x).cuda()
    out = plan.execute(d)
    assert worst_rel_l2(out.cpu().numpy(), ref, nx * ny) <= tol_fp32(nx * ny)
    plan.execute(d, out=d)
    assert worst_rel_l2(d.cpu().numpy(), ref, nx * ny) <= tol_fp32(nx * ny)
    plan.close()


@pytest.mark.parametrize("e", ["16", "32"])
@pytest.mark.parametrize("c,ny,nx,batch,split", [("2", 2048, 8, 2, "1"), ("2", 4096, 4, 1, "1"),
                                                 ("2", 8192, 16, 1, "2"), ("4", 4096, 4, 2, "1"),
                                                 ("4", 8192, 4, 1, "1"), ("4", 8192, 8, 1, "2")])
@pytest.mark.parametrize("inverse", [False, True])
def test_column_pass_by_dsmem_clusters(g, monkeypatch, e, c, ny, nx, batch, split, inverse):
    """Column pass by C-CTA clusters: each CTA stages 1/C of a column block with
    TMA, the radix-C combination reads the partners' slices through
    distributed shared memory; out of place and in place."""
    monkeypatch.setenv("GB300FFT_COL_CLUSTER", c)
    monkeypatch.setenv("GB300FFT_COL_E", e)
    monkeypatch.setenv("GB300FFT_SPLIT", split)
    plan = g.Plan(nx, ny, batch, inverse=inverse)
    for k in ("GB300FFT_COL_CLUSTER", "GB300FFT_COL_E", "GB300FFT_SPLIT"):
        monkeypatch.delenv(k)
    desc = plan.describe()
    if not desc["cols"]["kernel"].startswith("k_cols_cluster"):
        pytest.skip(f"no cluster variant for column block {desc['cols']['n']}")
    x = synth.uniform_complex((batch, ny, nx), seed=ny + 3 * nx + batch)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    d = torch.from_numpy(x).cuda()
    out = plan.execute(d)
    assert plan.status() == 0
    assert worst_rel_l2(out.cpu().numpy(), ref, nx * ny) <= tol_fp32(nx * ny)
    plan.execute(d, out=d)
    assert worst_rel_l2(d.cpu().numpy(), ref, nx * ny) <= tol_fp32(nx * ny)
    plan.close()


@pytest.mark.parametrize("e", ["16", "32", "64"])
@pytest.mark.parametrize("ny,nx,batch", [(4096, 4, 2), (4096, 64, 1), (8192, 8, 1), (8192, 2, 1)])
@pytest.mark.parametrize("inverse", [False, True])
def test_column_pass_elements_per_thread(g, monkeypatch, e, ny, nx, batch, inverse):
    """TMA column pass with 16, 32 or 64 elements per thread (one shared-memory
    exchange for a 4096-point column at E = 64); out of place and in place."""
    monkeypatch.setenv("GB300FFT_COL_E", e)
    plan = g.Plan(nx, ny, batch, inverse=inverse)
    monkeypatch.delenv("GB300FFT_COL_E")
    x = synth.uniform_complex((batch, ny, nx), seed=5 * ny + nx)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    d = torch.from_numpy(x).cuda()
    assert worst_rel_l2(plan.execute(d).cpu().numpy(), ref, nx * ny) <= tol_fp32(nx * ny)
    plan.execute(d, out=d)
    assert worst_rel_l2(d.cpu().numpy(), ref, nx * ny) <= tol_fp32(nx * ny)
    assert plan.status() == 0
    plan.close()


@pytest.mark.parametrize("ny,nx,batch", [(4096, 4, 2), (4096, 256, 1), (8192, 64, 1), (8192, 8192, 1),
                                         (8192, 8192, 2)])
@pytest.mark.parametrize("inverse", [False, True])
def test_streaming_column_pass_is_bit_identical(g, monkeypatch, ny, nx, batch, inverse):
    """The streaming column pass (row pass storing rows permuted, segments
    landing per warp) and the landed-pair row pass run the same operations in
    the same order as the plain row and column passes, so results agree bit
    for bit; both meet the oracle bound.  The batch of two 8192 x 8192
    transforms has pairs on both sides of the slice boundary."""
    monkeypatch.setenv("GB300FFT_COL_STREAM", "1")
    monkeypatch.setenv("GB300FFT_ROW_LAND", "1")
    ps = g.Plan(nx, ny, batch, inverse=inverse)
    monkeypatch.setenv("GB300FFT_COL_STREAM", "0")
    monkeypatch.setenv("GB300FFT_ROW_LAND", "0")
    pp = g.Plan(nx, ny, batch, inverse=inverse)
    monkeypatch.delenv("GB300FFT_COL_STREAM")
    monkeypatch.delenv("GB300FFT_ROW_LAND")
    if ny >= 8192 and nx == 8192:  # the landed-pair kernel serves 8192-point rows
        assert ps.describe()["rows"]["kernel"].startswith("k_rows_land<")
        assert pp.describe()["rows"]["kernel"].startswith("k_rows<")
    assert ps.describe()["cols"]["kernel"].startswith("k_cols_stream<")
    assert pp.describe()["cols"]["kernel"].startswith("k_cols<")
    x = synth.uniform_complex((batch, ny, nx), seed=7 * ny + nx)
    d = torch.from_numpy(x).cuda()
    a = ps.execute(d)
    b = pp.execute(d)
    torch.cuda.synchronize()
    assert ps.status() == 0 and pp.status() == 0
    assert torch.equal(torch.view_as_real(a), torch.view_as_real(b))
    # pre-split plans route the blocks through a planar workspace, so an
    # in-place call takes the same path and gives the same bits
    c = d.clone()
    ps.execute(c, out=c)
    torch.cuda.synchronize()
    if ny >= 8192:
        assert torch.equal(torch.view_as_real(c), torch.view_as_real(a))
    if nx * ny <= (1 << 20):
        ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
        assert worst_rel_l2(a.cpu().numpy(), ref, nx * ny) <= tol_fp32(nx * ny)
    ps.close()
    pp.close()


@pytest.mark.parametrize("nx,ny", [(8192, 8192), (1024, 1024)])
def test_pass_events_inside_a_captured_graph(g, nx, ny):
    """Steps captured into a CUDA graph (as bench.py times them) give the same
    result as eager calls, and their pass events, recorded as event-record
    nodes, time-stamp every replay: both passes take positive time and add
    up to no more than the whole replay."""
    x = torch.from_numpy(synth.normal_complex((ny, nx), seed=41)).cuda()
    plan = g.Plan(nx, ny, 1)
    ref = plan.execute(x).clone()
    out = torch.empty_like(x)
    plan.execute(x, out=out)  # warm-up: tensor maps cached before capture
    eager = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for e in eager:
        e.record()  # torch reads elapsed times only of events it has seen recorded
    plan.set_pass_events(*eager)  # outside capture: plain event records
    plan.execute(x, out=out)
    plan.set_pass_events(None, None, None)
    torch.cuda.synchronize()
    assert eager[0].elapsed_time(eager[1]) > 0 and eager[1].elapsed_time(eager[2]) > 0
    steps = 3
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for trip in evs:
        for e in trip:
            e.record()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for k in range(steps):
            plan.set_pass_events(*evs[k])
            plan.execute(x, out=out)
    plan.set_pass_events(None, None, None)
    out.zero_()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    graph.replay()
    b.record()
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(out, ref)
    total = a.elapsed_time(b)
    rows = [t[0].elapsed_time(t[1]) for t in evs]
    cols = [t[1].elapsed_time(t[2]) for t in evs]
    assert min(rows) > 0 and min(cols) > 0
    assert sum(rows) + sum(cols) <= total * 1.001


@pytest.mark.parametrize("n,batch", [(256, 1), (512, 1), (1024, 1), (512, 4), (256, 16)])
@pytest.mark.parametrize("inverse", [False, True])
def test_one_launch_small_arrays(g, monkeypatch, n, batch, inverse):
    """Small square arrays run rows and columns in one cooperative launch
    (grid barrier between the phases): against the oracle out of place and
    in place, equal to the two-launch form within the bound, and again when
    the calls are captured in a CUDA graph and replayed (the barrier resets
    itself each launch)."""
    plan = g.Plan(n, n, batch, inverse=inverse)
    assert plan.describe()["one_launch"] == 1
    monkeypatch.setenv("GB300FFT_SMALL2D", "0")
    two = g.Plan(n, n, batch, inverse=inverse)
    monkeypatch.delenv("GB300FFT_SMALL2D")
    assert two.describe()["one_launch"] == 0
    x = synth.uniform_complex((batch, n, n), seed=19 * n + batch)
    ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    d = torch.from_numpy(x).cuda()
    a = plan.execute(d).cpu().numpy()
    assert plan.status() == 0
    assert worst_rel_l2(a, ref, n * n) <= tol_fp32(n * n)
    assert worst_rel_l2(two.execute(d).cpu().numpy(), ref, n * n) <= tol_fp32(n * n)
    dd = d.clone()
    plan.execute(dd, out=dd)
    assert np.array_equal(dd.cpu().numpy(), a)
    out = torch.empty_like(d)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(3):
            plan.execute(d, out=out)
    for _ in range(2):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), a)
    assert plan.status() == 0
    plan.close()
    two.close()
