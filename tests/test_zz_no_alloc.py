"""fft_execute_ragged_noalloc: the ragged transform for callers that cannot
allocate device memory (graph capture in progress, memory owned by a pool or
framework allocator).  Its scratch is a fixed array inside the library; this
file checks it, through the C ABI, against the plan-based fft_execute_ragged.

Collected last (file name), so a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.helpers import rel_l2, tol_fp32

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_15437_gb300 import build
    build.build()
    from paper_2506_15437_gb300 import _native
    return _native.load()


def noalloc(lib, nx, ny, x, inverse=False, status=None):
    n = len(nx)
    ax = (ctypes.c_int * n)(*[int(v) for v in nx])
    ay = (ctypes.c_int * n)(*[int(v) for v in ny])
    out = torch.empty_like(x)
    rc = lib.fft_execute_ragged_noalloc(n, ax, ay, 1 if inverse else -1, x.data_ptr(), out.data_ptr(),
                                        status.data_ptr() if status is not None else None,
                                        torch.cuda.current_stream().cuda_stream)
    return rc, out


@pytest.mark.gpu
def test_noalloc_matches_plan_on_two_calls_in_a_row(lib):
    import paper_2506_15437_gb300 as g
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # two different batches back to back: the second call must not see the
    # first call's leftovers in the shared scratch array
    for seed, count, inverse in [(31, 96, False), (32, 40, True)]:
        nx, ny, offs, packed = synth.ragged_batch(count, seed=seed)
        x = torch.from_numpy(packed).cuda()
        rc, got = noalloc(lib, nx, ny, x, inverse=inverse, status=status)
        assert rc == 0
        ref = g.RaggedPlan(nx, ny, inverse=inverse).execute(x)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = got.cpu().numpy()
        ref = ref.cpu().numpy()
        for i in range(count):
            n = int(nx[i] * ny[i])
            assert rel_l2(got[offs[i]:offs[i] + n], ref[offs[i]:offs[i] + n]) <= tol_fp32(n), i


@pytest.mark.gpu
def test_noalloc_rejects_requests_beyond_its_fixed_scratch(lib):
    x = torch.zeros(1024 * 1024 * 8, dtype=torch.complex64, device="cuda")
    rc, _ = noalloc(lib, [32] * 1025, [32] * 1025, x)
    assert rc == -1  # FFT_ERR_INVALID_SIZE: more instances than the array holds
    big = [1024] * 300  # 300 instances of 1024 x 1024 need 76800 work items
    rc, _ = noalloc(lib, big, big, x)
    assert rc == -1
