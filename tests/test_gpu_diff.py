"""Differentiation form on the GPU: the hand-written adjoint behind
torch.autograd.Function, against the FP64 reference gradient
2 F^H (w (.) F x) (pinned against finite differences in test_diff_oracle.py)."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, rel_l2, tol_fp32

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


def ref_grad(x, w):
    X = oracle.fft2d(x, dir=-1, threads=ORACLE_THREADS)
    return 2.0 * oracle.fft2d(w * X, dir=1, threads=ORACLE_THREADS), np.sum(w * np.abs(X) ** 2)


@pytest.mark.parametrize("fused", [True, False])
def test_gradient_64x64_against_fp64(g, fused):
    n = 64
    x = synth.uniform_complex((n, n), seed=2506)
    w = synth.mask((n, n), seed=2507)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    wd = torch.from_numpy(w).cuda()
    if fused:
        L = g.weighted_power_loss(xd, wd)
    else:
        X = g.fft2(xd)
        L = (wd * (X.real ** 2 + X.imag ** 2)).sum()
    L.backward()
    gref, Lref = ref_grad(x, w)
    # two transforms (forward + adjoint): twice the single-transform bound
    assert rel_l2(xd.grad.cpu().numpy(), gref) <= 2 * tol_fp32(n * n)
    assert abs(L.item() - Lref) / Lref < 1e-5


def test_gradient_full_size_8x2048x2048(g):
    """x [8][2048][2048] U[-1,1), w U[0,1): fused forward + adjoint at full
    size, every slice of the gradient against the FP64 reference, and the
    loss against the FP64 loss."""
    b, n = 8, 2048
    x = synth.uniform_complex((b, n, n), seed=2506)
    w = synth.mask((b, n, n), seed=2507)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    wd = torch.from_numpy(w).cuda()
    L = g.weighted_power_loss(xd, wd)
    L.backward()
    grad = xd.grad.cpu().numpy()
    gref, Lref = ref_grad(x, w)
    worst = 0.0
    for k in range(b):
        e = rel_l2(grad[k], gref[k])
        worst = max(worst, e)
        assert e <= 2 * tol_fp32(n * n), k
    print(f"8 x 2048^2 gradient: worst per-slice rel L2 {worst:.3e}")
    assert abs(L.item() - Lref) / Lref < 1e-5


def test_fused_and_autograd_paths_agree(g):
    n = 512
    x = synth.uniform_complex((2, n, n), seed=5)
    w = synth.mask((2, n, n), seed=6)
    wd = torch.from_numpy(w).cuda()
    x1 = torch.from_numpy(x).cuda().requires_grad_(True)
    g.weighted_power_loss(x1, wd).backward()
    x2 = torch.from_numpy(x).cuda().requires_grad_(True)
    X = g.fft2(x2)
    (wd * (X.real ** 2 + X.imag ** 2)).sum().backward()
    assert rel_l2(x1.grad.cpu().numpy(), x2.grad.cpu().numpy()) <= 2 * tol_fp32(n * n)


def test_fft2_backward_is_adjoint_for_inverse_plans(g):
    """Gradient through an inverse transform: F^H of the inverse is the forward."""
    n = 128
    x = synth.uniform_complex((n, n), seed=9)
    c = synth.uniform_complex((n, n), seed=10)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    cd = torch.from_numpy(c).cuda()
    Y = g.fft2(xd, inverse=True)
    (Y.real * cd.real + Y.imag * cd.imag).sum().backward()
    # L = Re<c, F_inv x>: dL/dx (PyTorch convention) = F_inv^H c = F_fwd c
    ref = oracle.fft2d(c, dir=-1)
    assert rel_l2(xd.grad.cpu().numpy(), ref) <= tol_fp32(n * n)


def test_backward_reads_the_upstream_gradient_on_the_device(g):
    """WeightedPowerLoss.backward passes the upstream gradient to the adjoint
    as a device pointer: no host synchronisation inside autograd (torch's
    sync debug mode turns any into an error), and a non-unit upstream
    gradient scales the result exactly like the host-scale call."""
    n = 256
    x = synth.uniform_complex((2, n, n), seed=12)
    w = synth.mask((2, n, n), seed=13)
    wd = torch.from_numpy(w).cuda()
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    L = g.weighted_power_loss(xd, wd)
    out = 3.5 * L
    torch.cuda.synchronize()
    torch.cuda.set_sync_debug_mode("error")
    try:
        out.backward()
    finally:
        torch.cuda.set_sync_debug_mode(0)
    plan = g.get_plan(n, n, 2, False, "fp32", "cuda")
    # the loss runs the fused form here: its backward is the scaled row half
    assert plan.weighted_power_adjoint_parts() > 0
    _, y = plan.weighted_power_adjoint(torch.from_numpy(x).cuda(), wd)
    want = plan.backward_rows_scaled(y, None, 7.0)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(xd.grad), torch.view_as_real(want))
    gref, _ = ref_grad(x, w)
    assert rel_l2(xd.grad.cpu().numpy(), 3.5 * gref) <= 2 * tol_fp32(n * n)


def test_backward_weighted_dev_rejects_bad_scale_pointer(g):
    from paper_2506_15437_gb300 import _native as N
    n = 64
    plan = g.get_plan(n, n, 1, False, "fp32", "cuda")
    X = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    w = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    s = torch.zeros(2, dtype=torch.float32, device="cuda")
    lib = N.load()
    rc = lib.fft_backward_weighted_dev(plan._p, X.data_ptr(), w.data_ptr(), None, 1.0, X.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == N.FFT_ERR_INVALID_ARG
    rc = lib.fft_backward_weighted_dev(plan._p, X.data_ptr(), w.data_ptr(), s.data_ptr() + 2, 1.0, X.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == N.FFT_ERR_INVALID_ARG


# The fused form: fft_weighted_power_adjoint (forward rows, then one column
# pass that sums the loss and runs the adjoint's column half) and
# fft_backward_rows_scaled (the adjoint's row half).
FUSED_SHAPES = [(64, 64, 1), (256, 1024, 3), (1024, 256, 2), (2048, 2048, 1), (32, 4096, 1), (2048, 64, 2)]


@pytest.mark.parametrize("ny,nx,b", FUSED_SHAPES, ids=[f"{b}x{ny}x{nx}" for ny, nx, b in FUSED_SHAPES])
def test_fused_column_half_against_fp64(g, ny, nx, b):
    """y = F_cols^H (w (.) F x) against the FP64 oracle (the forward 2D
    transform, then the inverse-sign 1D transform down every column of the
    weighted product), the loss against sum w |F x|^2, and the full gradient
    2 F_rows^H y against 2 F^H (w (.) F x)."""
    x = synth.uniform_complex((b, ny, nx), seed=ny + 3 * nx + b)
    w = synth.mask((b, ny, nx), seed=ny + nx)
    plan = g.Plan(nx, ny, b)
    assert plan.weighted_power_adjoint_parts() > 0
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(w).cuda()
    L, y = plan.weighted_power_adjoint(xd, wd)
    G = plan.backward_rows_scaled(y, None, 2.0)
    torch.cuda.synchronize()
    assert plan.status() == 0
    X = oracle.fft2d(x, dir=-1, threads=ORACLE_THREADS)
    wx = w * X
    yref = np.swapaxes(oracle.fft1d_batch(np.ascontiguousarray(np.swapaxes(wx, -1, -2)), dir=1,
                                          threads=ORACLE_THREADS), -1, -2)
    n = nx * ny
    for k in range(b):
        assert rel_l2(y[k].cpu().numpy(), yref[k]) <= tol_fp32(n), k
    Lref = float(np.sum(w * np.abs(X) ** 2))
    assert abs(L.item() - Lref) / Lref < 1e-6
    gref, _ = ref_grad(x, w)
    for k in range(b):
        assert rel_l2(G[k].cpu().numpy(), gref[k]) <= 2 * tol_fp32(n), k
    plan.close()


def test_fused_and_unfused_forms_agree(g):
    """The same loss and gradient from both forms; in place (y over x) too."""
    n, b = 512, 2
    x = synth.uniform_complex((b, n, n), seed=41)
    w = synth.mask((b, n, n), seed=42)
    plan = g.Plan(n, n, b)
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(w).cuda()
    one = torch.ones(1, dtype=torch.float32, device="cuda")
    L1, y = plan.weighted_power_adjoint(xd, wd)
    G1 = plan.backward_rows_scaled(y, one, 2.0)
    X = plan.execute(xd)
    L2 = plan.weighted_power(X, wd)
    G2 = plan.backward_weighted_dev(X, wd, one, 2.0)
    torch.cuda.synchronize()
    assert abs(L1.item() - L2.item()) / L2.item() < 1e-6
    assert rel_l2(G1.cpu().numpy(), G2.cpu().numpy()) <= 2 * tol_fp32(n * n)
    d = xd.clone()
    L3, y3 = plan.weighted_power_adjoint(d, wd, d)
    assert y3.data_ptr() == d.data_ptr()
    assert L3.item() == L1.item() and torch.equal(torch.view_as_real(d), torch.view_as_real(y))
    G3 = plan.backward_rows_scaled(d, one, 2.0, out=d)
    assert torch.equal(torch.view_as_real(G3), torch.view_as_real(G1))
    plan.close()


def test_unfused_plans_keep_the_unfused_loss(g):
    """Inverse plans and columns longer than 2048 have no fused form: both
    calls report FFT_ERR_UNSUPPORTED, and the loss runs the unfused path
    with the same gradient bound."""
    from paper_2506_15437_gb300 import _native as N
    inv = g.Plan(64, 64, 1, inverse=True)
    assert inv.weighted_power_adjoint_parts() == 0
    assert inv._lib.fft_weighted_power_adjoint_parts(inv._p) == N.FFT_ERR_UNSUPPORTED
    z = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    assert inv._lib.fft_backward_rows_scaled(inv._p, z.data_ptr(), None, 1.0, z.data_ptr(), None) == \
        N.FFT_ERR_UNSUPPORTED
    inv.close()
    assert g.get_plan(16, 4096, 1, False, "fp32", "cuda").weighted_power_adjoint_parts() == 0
    ny, nx = 8192, 16
    long = g.get_plan(nx, ny, 1, False, "fp32", "cuda")
    assert long.weighted_power_adjoint_parts() == 0
    x = synth.uniform_complex((ny, nx), seed=51)
    w = synth.mask((ny, nx), seed=52)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    g.weighted_power_loss(xd, torch.from_numpy(w).cuda()).backward()
    gref, _ = ref_grad(x, w)
    assert rel_l2(xd.grad.cpu().numpy(), gref) <= 2 * tol_fp32(nx * ny)
