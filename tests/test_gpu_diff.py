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
    X = plan.execute(torch.from_numpy(x).cuda())
    want = plan.backward_weighted(X, wd, 7.0)
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
