"""Host-side arithmetic of bench.py (no GPU): the algorithmic bytes the
ragged form charges, and the whole-job throughput formula."""
import bench
import synth


def test_ragged_bytes_charge_one_pass_to_fused_instances():
    # 64 x 128 = 8192 points fit one CTA (one pass, 16 B/point); 128 x 128
    # needs rows then columns (two passes, 32 B/point)
    assert bench.ragged_algorithmic_bytes([64], [128]) == 16 * 8192
    assert bench.ragged_algorithmic_bytes([128], [128]) == 32 * 16384
    assert bench.ragged_algorithmic_bytes([32, 1024], [32, 1024]) == 16 * 1024 + 32 * 1024 * 1024


def test_ragged_bytes_of_the_benchmark_batch():
    nx, ny, _, packed = synth.ragged_batch(512, seed=2506)
    small = sum(int(a) * int(b) for a, b in zip(nx, ny) if a * b <= 8192)
    assert bench.ragged_algorithmic_bytes(nx, ny) == 32.0 * packed.size - 16.0 * small
    assert small > 0


def test_job_gflops_is_whole_job():
    # 2 ranks, each 1 GFLOP in 1 ms -> 2000 GFLOP/s for the job
    assert abs(bench.job_gflops(2, 1e9, 1.0) - 2000.0) < 1e-9
