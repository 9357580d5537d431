"""Ragged batches (many 2D transforms of mixed sizes, one persistent launch
from a CUDA graph) against the FP64 oracle, instance by instance."""
import os

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


def check_instances(nx, ny, offs, packed, got, inverse=False):
    worst = 0.0
    for i in range(len(nx)):
        n = int(nx[i] * ny[i])
        x = packed[offs[i]:offs[i] + n].reshape(ny[i], nx[i])
        ref = oracle.fft2d(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
        err = rel_l2(got[offs[i]:offs[i] + n].reshape(ny[i], nx[i]), ref)
        assert err <= tol_fp32(n), (i, nx[i], ny[i], err)
        worst = max(worst, err)
    return worst


def run(g, nx, ny, packed, inverse=False, loop=False):
    plan = g.RaggedPlan(nx, ny, inverse=inverse)
    d = torch.from_numpy(packed).cuda()
    out = plan.execute_loop(d) if loop else plan.execute(d)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return plan, out.cpu().numpy()


def test_ragged_512_batch(g):
    """512 instances, each axis log-uniform on 32..1024, seed 2506."""
    nx, ny, offs, packed = synth.ragged_batch(512, seed=2506)
    plan, got = run(g, nx, ny, packed)
    for i in range(0, 512, 37):
        assert plan.offset(i) == offs[i]
    assert plan.total == packed.size
    check_instances(nx, ny, offs, packed, got)


@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("seed", [1, 2])
def test_ragged_mixed_small(g, inverse, seed):
    nx, ny, offs, packed = synth.ragged_batch(40, seed=seed)
    _, got = run(g, nx, ny, packed, inverse=inverse)
    check_instances(nx, ny, offs, packed, got, inverse=inverse)


@pytest.mark.parametrize("shapes", [
    [(32, 32)],                       # one fused instance
    [(1024, 1024)],                   # one large instance
    [(1024, 32), (32, 1024)],         # extreme aspect ratios, row/column items
    [(32, 64), (64, 32), (32, 128), (128, 32), (64, 64)],  # every fused shape class (at most 4096 points)
    [(256, 32), (32, 256), (64, 128), (128, 64)],  # 8192 points: row and column items
    [(512, 512)] * 3 + [(32, 32)] * 5,
])
def test_ragged_shape_classes(g, shapes):
    nx = np.array([s[0] for s in shapes])
    ny = np.array([s[1] for s in shapes])
    sizes = nx * ny
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    packed = synth.uniform_complex((int(sizes.sum()),), seed=int(sizes.sum()))
    _, got = run(g, nx, ny, packed)
    check_instances(nx, ny, offs, packed, got)


def test_graph_replay_is_repeatable_and_matches_loop(g):
    nx, ny, offs, packed = synth.ragged_batch(64, seed=5)
    plan = g.RaggedPlan(nx, ny)
    d = torch.from_numpy(packed).cuda()
    a = plan.execute(d).clone()
    b = plan.execute(d).clone()
    c = plan.execute_loop(d)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    for i in range(len(nx)):
        n = int(nx[i] * ny[i])
        assert rel_l2(a[offs[i]:offs[i] + n].cpu().numpy(), c[offs[i]:offs[i] + n].cpu().numpy()) <= tol_fp32(n)


def test_ragged_in_place(g):
    nx, ny, offs, packed = synth.ragged_batch(24, seed=8)
    plan = g.RaggedPlan(nx, ny)
    d = torch.from_numpy(packed).cuda()
    plan.execute(d, out=d)
    torch.cuda.synchronize()
    check_instances(nx, ny, offs, packed, d.cpu().numpy())


def test_ragged_autotuned_schedule_is_correct(g, monkeypatch):
    monkeypatch.setenv("GB300FFT_AUTOTUNE", "1")
    nx, ny, offs, packed = synth.ragged_batch(48, seed=12)
    plan = g.RaggedPlan(nx, ny)
    monkeypatch.delenv("GB300FFT_AUTOTUNE")
    got = plan.execute(torch.from_numpy(packed).cuda()).cpu().numpy()
    assert plan.status() == 0
    check_instances(nx, ny, offs, packed, got)


def test_bounded_wait_reports_timeout(g, monkeypatch):
    """Failure detection without a GPU fault: a host-side test hook makes row
    items skip their completion count, so every column item's bounded wait
    runs out (after 2 ms); the kernel records FFT_ERR_TIMEOUT and returns, and
    the context stays usable for the next plan."""
    monkeypatch.setenv("GB300FFT_DEBUG_WITHHOLD", "1")
    monkeypatch.setenv("GB300FFT_SPIN_LIMIT_NS", "2000000")
    nx, ny = [512, 1024], [1024, 512]
    plan = g.RaggedPlan(nx, ny)
    monkeypatch.delenv("GB300FFT_DEBUG_WITHHOLD")
    monkeypatch.delenv("GB300FFT_SPIN_LIMIT_NS")
    x = torch.zeros(plan.total, dtype=torch.complex64, device="cuda")
    plan.execute(x)
    torch.cuda.synchronize()
    from paper_2506_15437_gb300 import _native as N
    assert plan.status() == N.FFT_ERR_TIMEOUT
    assert plan.status() == 0  # reading the status clears it
    plan.close()
    # the device still works
    nx2, ny2, offs2, packed2 = synth.ragged_batch(4, seed=3)
    _, got = run(g, nx2, ny2, packed2)
    check_instances(nx2, ny2, offs2, packed2, got)
