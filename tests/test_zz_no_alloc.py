"""fft_execute_ragged_noalloc: the ragged transform for callers that cannot
allocate device memory (a process whose device memory belongs to a pool or
framework allocator it must not go around, or a runtime that forbids device
allocation after start-up).  Its scratch is a fixed array inside the
library.  These tests call it through the C ABI and compare it with the
plan-based fft_execute_ragged (same kernel, plan-owned scratch) and with the
FP64 oracle, instance by instance.

Collected last (file name), so a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, rel_l2, tol_fp32

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_15437_gb300 import build
    build.build()
    from paper_2506_15437_gb300 import _native
    return _native.load()


def noalloc(lib, nx, ny, x, inverse=False, status=None, out=None):
    n = len(nx)
    ax = (ctypes.c_int * n)(*[int(v) for v in nx])
    ay = (ctypes.c_int * n)(*[int(v) for v in ny])
    if out is None:
        out = torch.empty_like(x)
    rc = lib.fft_execute_ragged_noalloc(n, ax, ay, 1 if inverse else -1, x.data_ptr(), out.data_ptr(),
                                        status.data_ptr() if status is not None else None,
                                        torch.cuda.current_stream().cuda_stream)
    return rc, out


def check_instances(got, ref, nx, ny, offs):
    for i in range(len(nx)):
        n = int(nx[i] * ny[i])
        assert rel_l2(got[offs[i]:offs[i] + n], ref[offs[i]:offs[i] + n]) <= tol_fp32(n), i


def oracle_packed(packed, nx, ny, offs, inverse):
    ref = np.empty(packed.shape, np.complex128)
    for i in range(len(nx)):
        a, n = offs[i], int(nx[i] * ny[i])
        ref[a:a + n] = oracle.fft2d(packed[a:a + n].reshape(int(ny[i]), int(nx[i])),
                                    dir=1 if inverse else -1, threads=ORACLE_THREADS).ravel()
    return ref


@pytest.mark.gpu
def test_noalloc_matches_plan_and_oracle_on_two_calls_in_a_row(lib):
    import paper_2506_15437_gb300 as g
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # two different batches back to back: the second call must not see the
    # first call's leftovers in the shared scratch array
    for seed, count, inverse in [(31, 96, False), (32, 40, True)]:
        nx, ny, offs, packed = synth.ragged_batch(count, seed=seed)
        x = torch.from_numpy(packed).cuda()
        rc, got = noalloc(lib, nx, ny, x, inverse=inverse, status=status)
        assert rc == 0
        plan = g.RaggedPlan(nx, ny, inverse=inverse)
        ref = plan.execute(x)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = got.cpu().numpy()
        check_instances(got, ref.cpu().numpy(), nx, ny, offs)
        check_instances(got, oracle_packed(packed, nx, ny, offs, inverse), nx, ny, offs)
        plan.close()


@pytest.mark.gpu
def test_noalloc_in_place(lib):
    """in == out: the same kernel reads each instance's pass input before any
    pass of that instance writes over it."""
    import paper_2506_15437_gb300 as g
    nx, ny, offs, packed = synth.ragged_batch(64, seed=33)
    x = torch.from_numpy(packed).cuda()
    plan = g.RaggedPlan(nx, ny)
    ref = plan.execute(x).cpu().numpy()
    d = x.clone()
    rc, out = noalloc(lib, nx, ny, d, out=d)
    assert rc == 0 and out.data_ptr() == d.data_ptr()
    torch.cuda.synchronize()
    check_instances(d.cpu().numpy(), ref, nx, ny, offs)
    check_instances(d.cpu().numpy(), oracle_packed(packed, nx, ny, offs, False), nx, ny, offs)
    plan.close()


@pytest.mark.gpu
def test_noalloc_leaves_a_set_status_word_alone(lib):
    """The kernel only ever records a failure into a status word that still
    reads 0; a word the caller already set keeps its value."""
    nx, ny, offs, packed = synth.ragged_batch(16, seed=34)
    x = torch.from_numpy(packed).cuda()
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    rc, got = noalloc(lib, nx, ny, x, status=status)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 7
    check_instances(got.cpu().numpy(), oracle_packed(packed, nx, ny, offs, False), nx, ny, offs)


@pytest.mark.gpu
def test_noalloc_rejects_requests_beyond_its_fixed_scratch(lib):
    x = torch.zeros(1024 * 1024 * 8, dtype=torch.complex64, device="cuda")
    rc, _ = noalloc(lib, [32] * 1025, [32] * 1025, x)
    assert rc == -1  # FFT_ERR_INVALID_SIZE: more instances than the array holds
    big = [1024] * 300  # 300 instances of 1024 x 1024 need 153600 work items
    rc, _ = noalloc(lib, big, big, x)
    assert rc == -1
