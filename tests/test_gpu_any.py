"""GPU parity of transforms whose sizes are not powers of two (Bluestein
over the power-of-two path, transposes for the y axis) against the FP64
any-length oracle, through the C ABI via the ctypes binding.

Bar: relative L2 error per transform <= tol_any (tests/helpers.py: the
power-of-two bound per power-of-two axis, 2e-7 * (3 log2 M + 3) per
Bluestein axis of padded length M, added over the axes).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, tol_any, worst_rel_l2

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


LENGTHS_1D = [3, 5, 6, 7, 12, 15, 31, 100, 127, 1000, 1536, 3000, 4095, 8191, 10007, 65535]


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
             (64, 6), (1, 1000), (1000, 1)]


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


def test_long_1d_million_points(g):
    n = 1_000_000  # 2^6 * 5^6: Bluestein over the four-step path (M = 2^21)
    x = synth.uniform_complex((1, n), seed=2506)
    plan = g.get_plan(n, 1, 1, False, "fp32", "cuda")
    assert plan.describe()["x"]["bluestein_m"] == 1 << 21
    got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fft1d_any(x, threads=ORACLE_THREADS)
    assert worst_rel_l2(got, ref, n) <= tol_any(n, 1)


@pytest.mark.parametrize("n", [5, 100, 1000, 4095])
def test_fused_and_unfused_bluestein_agree(g, monkeypatch, n):
    """Padded lengths up to 8192 run the fused kernels (chirp and filter
    products inside the two transforms); both forms meet the bound and agree
    closely (the same arithmetic in a different grouping of passes)."""
    x = synth.uniform_complex((3, n), seed=77 + n)
    fused = g.Plan(n, 1, 3)
    assert fused.describe()["x"]["fused"] == 1
    monkeypatch.setenv("GB300FFT_BLUESTEIN_FUSED", "0")
    plain = g.Plan(n, 1, 3)
    monkeypatch.delenv("GB300FFT_BLUESTEIN_FUSED")
    assert plain.describe()["x"]["fused"] == 0
    d = torch.from_numpy(x).cuda()
    a = fused.execute(d).cpu().numpy()
    b = plain.execute(d).cpu().numpy()
    ref = oracle.fft1d_any(x, threads=ORACLE_THREADS)
    assert worst_rel_l2(a, ref, n) <= tol_any(n, 1)
    assert worst_rel_l2(b, ref, n) <= tol_any(n, 1)
    fused.close()
    plain.close()


def test_describe_and_unsupported(g):
    plan = g.get_plan(1000, 3, 1, False, "fp32", "cuda")
    d = plan.describe()
    assert d["kind"] == "any" and d["x"]["bluestein_m"] == 2048 and d["y"]["bluestein_m"] == 8
    assert d["transposes"] == 2
    X = torch.zeros(3000, dtype=torch.complex64, device="cuda")
    w = torch.zeros(3000, dtype=torch.float32, device="cuda")
    with pytest.raises(g.FFTError):
        plan.backward_weighted(X, w, 2.0)
    with pytest.raises(g.FFTError):
        g.Plan(1000, 3, 1, precision="split_tc")
