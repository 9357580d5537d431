"""Dense-plan autotuner: picks a schedule by timing, stays correct, and
writes/reads its on-disk cache."""
import json

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, tol_fp32, worst_rel_l2

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


@pytest.mark.parametrize("ny,nx,batch", [(2048, 512, 1), (512, 4096, 2), (1, 8192, 64)])
def test_autotune_correct_and_cached(g, tmp_path, monkeypatch, ny, nx, batch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("GB300FFT_TUNE_CACHE", str(cache))
    plan = g.Plan(nx, ny, batch)
    plan.autotune()
    tuned = plan.describe()
    x = synth.uniform_complex((batch, ny, nx), seed=nx + ny)
    ref = oracle.fft2d(x, threads=ORACLE_THREADS)
    got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    assert worst_rel_l2(got, ref, nx * ny) <= tol_fp32(nx * ny)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])
    assert entry["key"].startswith(f"{nx}x{ny}x{batch}:0:")
    # a new plan of the same shape reads the cache and runs the same schedule
    again = g.Plan(nx, ny, batch)
    assert again.describe() == tuned
    plan.close()
    again.close()
