"""GPU parity of transforms whose sizes are not powers of two (mixed-radix
stages for 13-smooth lengths, Bluestein over the power-of-two path for the
rest) against the FP64 any-length oracle, through the C ABI via the ctypes
binding.

Bar: relative L2 error per transform <= tol_any (tests/helpers.py: the
power-of-two bound per power-of-two axis, 2e-7 * (log2 n + odd prime
factors) per mixed-radix axis, 2e-7 * (3 log2 M + 3) per Bluestein axis of
padded length M, added over the axes).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, mixed_eligible, mixed_fourstep_eligible, tol_any, worst_rel_l2

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


LENGTHS_1D = [3, 5, 6, 7, 12, 15, 17, 31, 100, 127, 1000, 1536, 3000, 4093, 4095, 8191, 10007, 65535]


@pytest.mark.parametrize("n", LENGTHS_1D)
@pytest.mark.parametrize("inverse", [False, True])
def test_1d_any_length(g, n, inverse):
    batch = 3 if n < 10000 else 1
    x = synth.uniform_complex((batch, n), seed=900 + n)
    plan = g.get_plan(n, 1, batch, inverse, "fp32", "cuda")
    got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    ref = oracle.fft1d_any(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    assert worst_rel_l2(got, ref, n) <= tol_any(n, 1), n


SHAPES_2D = [(3, 5), (12, 7), (100, 60), (60, 100), (1000, 3), (3, 1000), (480, 720), (256, 100), (100, 256),
             (64, 6), (1, 1000), (1000, 1), (16384, 4), (4, 16384), (2, 32768), (16384, 3)]


@pytest.mark.parametrize("ny,nx", SHAPES_2D, ids=[f"{a}x{b}" for a, b in SHAPES_2D])
@pytest.mark.parametrize("inverse", [False, True])
def test_2d_any_shape(g, ny, nx, inverse):
    x = synth.uniform_complex((2, ny, nx), seed=31 * nx + ny)
    plan = g.get_plan(nx, ny, 2, inverse, "fp32", "cuda")
    got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    ref = oracle.fft2d_any(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    assert worst_rel_l2(got, ref, nx * ny) <= tol_any(nx, ny), (ny, nx)


def test_in_place_and_backward(g):
    ny, nx = 300, 200
    x = synth.uniform_complex((ny, nx), seed=4)
    plan = g.get_plan(nx, ny, 1, False, "fp32", "cuda")
    d = torch.from_numpy(x).cuda()
    plan.execute(d, out=d)
    ref = oracle.fft2d_any(x, threads=ORACLE_THREADS)
    assert worst_rel_l2(d.cpu().numpy(), ref, nx * ny) <= tol_any(nx, ny)
    gy = synth.uniform_complex((ny, nx), seed=5)
    got = plan.backward(torch.from_numpy(gy).cuda()).cpu().numpy()
    assert worst_rel_l2(got, oracle.fft2d_any(gy, dir=1, threads=ORACLE_THREADS), nx * ny) <= tol_any(nx, ny)


def test_fft2_autograd_any_shape(g):
    ny, nx = 90, 70
    x = torch.from_numpy(synth.uniform_complex((ny, nx), seed=8)).cuda().requires_grad_(True)
    w = torch.from_numpy(synth.mask((ny, nx), seed=9)).cuda()
    X = g.fft2(x)
    (w * (X.real ** 2 + X.imag ** 2)).sum().backward()
    wX = w.cpu().numpy() * X.detach().cpu().numpy().astype(np.complex128)
    ref = 2.0 * oracle.fft2d_any(wX, dir=1, threads=ORACLE_THREADS)
    assert worst_rel_l2(x.grad.cpu().numpy(), ref, nx * ny) <= 2 * tol_any(nx, ny)


def test_long_1d_million_points(g, monkeypatch):
    """10^6 = 2^6 5^6: the mixed-radix four-step (1000 x 1000); with mixed
    radix switched off, Bluestein over the power-of-two four-step path
    (M = 2^21)."""
    n = 1_000_000
    x = synth.uniform_complex((1, n), seed=2506)
    ref = oracle.fft1d_any(x, threads=ORACLE_THREADS)
    plan = g.Plan(n, 1, 1)
    assert plan.describe()["x"]["mixed_fourstep"] == [1000, 1000]
    got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert worst_rel_l2(got, ref, n) <= tol_any(n, 1)
    monkeypatch.setenv("GB300FFT_MIXED", "0")
    blu = g.Plan(n, 1, 1)
    monkeypatch.delenv("GB300FFT_MIXED")
    assert blu.describe()["x"]["bluestein_m"] == 1 << 21
    got = blu.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert worst_rel_l2(got, ref, n) <= tol_any(n, 1, mixed=False)
    plan.close()
    blu.close()


# Smooth lengths beyond one CTA: the mixed-radix four-step.  Prime powers
# (5^7, 7^6, 3^10, 13^5), a power of two times 3, 15 and 9 stages, 11 and
# 13 stages on both passes, and the longest balanced case below 2^24.
MIXED_FS = [(15360, 3), (20000, 2), (78125, 2), (117649, 1), (59049, 1), (13 ** 5, 1), (1001 * 1000, 1),
            (3 << 20, 1), (2 ** 9 * 3 ** 9, 1)]


@pytest.mark.parametrize("n,batch", MIXED_FS, ids=[f"{a}x{b}" for a, b in MIXED_FS])
@pytest.mark.parametrize("inverse", [False, True])
def test_mixed_radix_fourstep(g, n, batch, inverse):
    assert mixed_fourstep_eligible(n)
    x = synth.uniform_complex((batch, n), seed=n % 9973)
    plan = g.Plan(n, 1, batch, inverse=inverse)
    n1, n2 = plan.describe()["x"]["mixed_fourstep"]
    assert n1 * n2 == n and max(n1, n2) <= 14336
    d = torch.from_numpy(x).cuda()
    got = plan.execute(d).cpu().numpy()
    ref = oracle.fft1d_any(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    err = worst_rel_l2(got, ref, n)
    print(f"mixedfs n={n} ({n1}x{n2}) inverse={inverse} err={err:.3e} tol={tol_any(n, 1):.3e}")
    assert err <= tol_any(n, 1), n
    plan.execute(d, out=d)  # in place: the first pass reads the input, the second writes it
    assert np.array_equal(d.cpu().numpy(), got)
    assert plan.status() == 0
    plan.close()


@pytest.mark.parametrize("n", [5, 100, 1000, 4095, 2049, 3])
@pytest.mark.parametrize("inverse", [False, True])
def test_fused_and_unfused_bluestein_agree(g, monkeypatch, n, inverse):
    """Padded lengths up to 8192 run the fused kernels: by default one pass
    (the forward transform's outputs stay in registers, times the filter,
    into the inverse), else two passes through the padded rows (chirp and
    filter products inside the two transforms), else five.  Every form meets
    the bound against the oracle; the one-pass form also in place."""
    x = synth.uniform_complex((3, n), seed=77 + n)
    monkeypatch.setenv("GB300FFT_MIXED", "0")  # smooth lengths take Bluestein too
    default = g.Plan(n, 1, 3, inverse=inverse)
    M = default.describe()["x"]["bluestein_m"]
    assert default.describe()["x"]["fused"] == (2 if M <= 2048 else 1)  # the faster form per padded length
    default.close()
    monkeypatch.setenv("GB300FFT_BLUESTEIN_ONEPASS", "1")
    one = g.Plan(n, 1, 3, inverse=inverse)
    assert one.describe()["x"]["fused"] == 2
    monkeypatch.setenv("GB300FFT_BLUESTEIN_ONEPASS", "0")
    two = g.Plan(n, 1, 3, inverse=inverse)
    monkeypatch.delenv("GB300FFT_BLUESTEIN_ONEPASS")
    assert two.describe()["x"]["fused"] == 1
    monkeypatch.setenv("GB300FFT_BLUESTEIN_FUSED", "0")
    plain = g.Plan(n, 1, 3, inverse=inverse)
    monkeypatch.delenv("GB300FFT_BLUESTEIN_FUSED")
    monkeypatch.delenv("GB300FFT_MIXED")
    assert plain.describe()["x"]["fused"] == 0
    d = torch.from_numpy(x).cuda()
    ref = oracle.fft1d_any(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    for plan in (one, two, plain):
        got = plan.execute(d).cpu().numpy()
        assert plan.status() == 0
        assert worst_rel_l2(got, ref, n) <= tol_any(n, 1, mixed=False), plan.describe()["x"]["fused"]
    a = one.execute(d).cpu().numpy()
    one.execute(d, out=d)  # in place: each CTA reads its rows before it writes them
    assert np.array_equal(d.cpu().numpy(), a)
    for plan in (one, two, plain):
        plan.close()


def test_describe_and_unsupported(g):
    plan = g.get_plan(1003, 17, 1, False, "fp32", "cuda")  # 17 * 59 and 17: Bluestein both ways
    d = plan.describe()
    assert d["kind"] == "any" and d["x"]["bluestein_m"] == 2048 and d["y"]["bluestein_m"] == 64
    assert d["x"]["mixed"] == 0 and d["transposes"] == 2
    assert g.get_plan(1001, 11, 1, False, "fp32", "cuda").describe()["x"]["mixed"] == 1  # 7 * 11 * 13
    X = torch.zeros(17051, dtype=torch.complex64, device="cuda")
    w = torch.zeros(17051, dtype=torch.float32, device="cuda")
    with pytest.raises(g.FFTError):
        plan.backward_weighted(X, w, 2.0)
    with pytest.raises(g.FFTError):
        g.Plan(1000, 3, 1, precision="split_tc")
    m = g.get_plan(1000, 3, 1, False, "fp32", "cuda").describe()
    assert m["x"]["mixed"] == 1 and m["y"]["mixed"] == 1 and m["x"]["bluestein_m"] == 0
    assert m["transposes"] == 0  # the y axis runs down the columns in place


# Mixed-radix lengths: every radix alone and in combination (16, 8, 4, 2,
# the two-level 15, 14, 12, 10, 9 and 6, the single 3, 5, 7, 11, 13), prime
# powers, the longest length, and short rows packed several to a CTA.
MIXED_1D = [3, 5, 6, 7, 9, 10, 11, 12, 13, 14, 15, 21, 24, 25, 35, 45, 49, 60, 96, 100, 105, 120, 135, 143, 196,
            210, 225, 343, 360, 405, 625, 1000, 1001, 1080, 1125, 1728, 1920, 2025, 2187, 2197, 2744, 3125, 3375,
            4095, 6000, 7168, 10000, 12288, 13312, 14080, 14336]


@pytest.mark.parametrize("n", MIXED_1D)
@pytest.mark.parametrize("inverse", [False, True])
def test_mixed_radix_1d(g, n, inverse):
    assert mixed_eligible(n)
    batch = 3 if n > 64 else 131  # short rows: several CTAs, the last one partly filled
    x = synth.uniform_complex((batch, n), seed=1300 + n)
    plan = g.Plan(n, 1, batch, inverse=inverse)
    assert plan.describe()["x"]["mixed"] == 1
    d = torch.from_numpy(x).cuda()
    got = plan.execute(d).cpu().numpy()
    ref = oracle.fft1d_any(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    err = worst_rel_l2(got, ref, n)
    print(f"mixed1d n={n} inverse={inverse} err={err:.3e} tol={tol_any(n, 1):.3e}")
    assert err <= tol_any(n, 1), n
    plan.execute(d, out=d)  # in place: every CTA reads its rows before writing them
    assert np.array_equal(d.cpu().numpy(), got)
    assert plan.status() == 0
    plan.close()


# (ny, nx): y by the column kernel with 8, 4, 2 or 1 adjacent columns (odd
# nx), x mixed or a power of two or Bluestein, y longest at 14336; axes
# longer than 14336 by the four-step form (x directly, y between transposes)
MIXED_2D = [(1000, 1000), (1080, 1920), (7, 1024), (100, 61), (61, 100), (1024, 7), (14336, 8), (12, 14336),
            (9, 6), (3, 5), (600, 2), (3, 20000), (15360, 2), (1001, 143), (13, 4095)]


@pytest.mark.parametrize("ny,nx", MIXED_2D, ids=[f"{a}x{b}" for a, b in MIXED_2D])
@pytest.mark.parametrize("inverse", [False, True])
def test_mixed_radix_2d(g, ny, nx, inverse):
    batch = 2
    x = synth.uniform_complex((batch, ny, nx), seed=17 * nx + ny)
    plan = g.Plan(nx, ny, batch, inverse=inverse)
    desc = plan.describe()
    assert desc["y"]["mixed"] == (1 if mixed_eligible(ny) else 0)
    assert desc["transposes"] == (0 if mixed_eligible(ny) else 2)
    d = torch.from_numpy(x).cuda()
    got = plan.execute(d).cpu().numpy()
    ref = oracle.fft2d_any(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    err = worst_rel_l2(got, ref, nx * ny)
    print(f"mixed2d {ny}x{nx} inverse={inverse} err={err:.3e} tol={tol_any(nx, ny):.3e}")
    assert err <= tol_any(nx, ny), (ny, nx)
    plan.execute(d, out=d)
    assert np.array_equal(d.cpu().numpy(), got)
    assert plan.status() == 0
    plan.close()


@pytest.mark.parametrize("ny,nx", [(1, 1000), (1000, 1000), (360, 210)])
def test_mixed_radix_and_bluestein_agree(g, monkeypatch, ny, nx):
    """The same smooth sizes through Bluestein (mixed radix switched off):
    both meet their bounds against the oracle."""
    x = synth.uniform_complex((ny, nx), seed=5 * nx + ny)
    d = torch.from_numpy(x).cuda()
    mixed = g.Plan(nx, ny, 1)
    monkeypatch.setenv("GB300FFT_MIXED", "0")
    blu = g.Plan(nx, ny, 1)
    monkeypatch.delenv("GB300FFT_MIXED")
    assert mixed.describe()["x"]["mixed"] == 1 and blu.describe()["x"]["mixed"] == 0
    ref = (oracle.fft1d_any(x, threads=ORACLE_THREADS) if ny == 1
           else oracle.fft2d_any(x, threads=ORACLE_THREADS))
    assert worst_rel_l2(mixed.execute(d).cpu().numpy(), ref, nx * ny) <= tol_any(nx, ny)
    assert worst_rel_l2(blu.execute(d).cpu().numpy(), ref, nx * ny) <= tol_any(nx, ny, mixed=False)
    mixed.close()
    blu.close()


# The bench's any-size batches at their full sizes and in their launch
# configuration (one plan over the whole batch): 64 sampled signals of each
# against the oracle, the rest through properties that hold at any size.
BENCH_1D = [(3000, 16384), (4095, 16384), (4093, 16384), (1001, 32768), (1_000_000, 32)]


@pytest.mark.parametrize("n,batch", BENCH_1D, ids=[f"{n}x{b}" for n, b in BENCH_1D])
def test_bench_batches_full_size_sampled(g, n, batch):
    x = synth.uniform_complex((batch, n), seed=2506 + n)
    plan = g.Plan(n, 1, batch)
    d = plan.describe()["x"]
    assert (d["bluestein_m"] > 0) == (n == 4093)  # the prime takes Bluestein, the smooth lengths mixed radix
    dx = torch.from_numpy(x).cuda()
    got = plan.execute(dx)
    torch.cuda.synchronize()
    assert plan.status() == 0
    rows = np.unique(np.concatenate([[0, batch - 1], np.random.default_rng(n).integers(0, batch, 62 if n < 10 ** 5 else 2)]))
    ref = oracle.fft1d_any(x[rows], threads=ORACLE_THREADS)
    err = worst_rel_l2(got[torch.from_numpy(rows).cuda()].cpu().numpy(), ref, n)
    print(f"bench batch {batch}x{n}: {len(rows)} sampled signals, worst rel L2 {err:.3e} (bound {tol_any(n, 1):.2e})")
    assert err <= tol_any(n, 1), (n, err)
    # every signal: Parseval (sum |X|^2 = n sum |x|^2), and the inverse plan
    # brings back n x
    e_in = (dx.abs() ** 2).sum(dim=1).double()
    e_out = (got.abs() ** 2).sum(dim=1).double() / n
    assert torch.max(torch.abs(e_out / e_in - 1)).item() <= 20 * tol_any(n, 1)
    inv = g.Plan(n, 1, batch, inverse=True)
    back = inv.execute(got) / n
    rt = (torch.linalg.vector_norm(back - dx, dim=1) / torch.linalg.vector_norm(dx, dim=1)).max().item()
    assert rt <= 2 * tol_any(n, 1), rt
    for p in (plan, inv):
        p.close()


@pytest.mark.parametrize("first", [1000, 4095])
def test_mixed_plans_with_different_shared_memory_coexist(g, first):
    """Two mixed-radix plans whose CTAs need different amounts of dynamic
    shared memory above 48 KiB from the same kernel (1000-point rows four to
    a CTA, one 4095-point row per CTA), created one after the other: the
    later plan must not leave the kernel unable to launch the earlier one's
    CTAs (it did when each plan set the kernel's limit to its own size)."""
    shapes = {1000: 8, 4095: 2}
    order = [first, 4095 if first == 1000 else 1000]
    plans = {n: g.Plan(n, 1, shapes[n]) for n in order}
    for n in order + order:
        x = synth.uniform_complex((shapes[n], n), seed=n)
        got = plans[n].execute(torch.from_numpy(x).cuda()).cpu().numpy()
        assert plans[n].status() == 0
        assert worst_rel_l2(got, oracle.fft1d_any(x, threads=ORACLE_THREADS), n) <= tol_any(n, 1), n
    for p in plans.values():
        p.close()
