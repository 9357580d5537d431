"""Throughput of the gb300fft hot path on GB300.

Headline workload: one forward 2D complex64 FFT of 8192 x 8192 (inputs
N(0,1) re/im, seed 2506) on the plain FP32 path -- the largest configuration
of the square-size sweep, and the one the HBM-roofline target is stated on.
A step is one fft_execute over the whole array (row pass + column pass, the
twiddles and the reorders fused in).  Input and output are 512 MiB each, far
larger than L2, so no flush is needed between steps.

Metric: GFLOP/s under the 5 N log2 N convention (N = nx*ny per transform),
whole-job over all ranks.  Beside it: the roofline of the dominant kernel
(algorithmic bytes / CUDA-event duration, measured live on the launching
stream), an end-to-end figure with pinned host buffers and the copies inside
the timed region, the FP64 CPU oracle timed on a bounded sample, and the
other forms (inverse, other sizes, split tensor-core, differentiation,
ragged batch) in "forms".

  python bench.py [--gpus N --steps K --warmup W]      # this library
  python bench.py --impl reference [...]               # the FP64 CPU oracle
Multi-GPU: launched by torchrun, one rank per GPU, independent replicas
(weak scaling; the batched/2D transform needs no exchange per rank).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "2D C2C FFT GFLOP/s (5N log2N), % of HBM roofline; split-TC vs FP32 path"
NX = NY = 8192
SEED = 2506


def flops_2d(nx, ny, batch=1):
    n = nx * ny
    return 5.0 * n * math.log2(n) * batch if n > 1 else 0.0


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured", d
    return 6800.0, "fallback", {}


def read_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    return None if e is None else float(e["bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        t0, t1 = (self.marks[0], self.marks[-1]) if len(self.marks) >= 2 else (0, 1e18)
        inside = [s for t, s in self.samples if t0 - 0.15 <= t <= t1 + 0.15] or [s for _, s in self.samples[-3:]]
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in inside:
            f = [x.strip() for x in s.split(",")]
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(inside)}


def max_over_ranks(dist, value: float, device) -> float:
    """Largest `value` over all ranks (the step time every rank reports)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(world: int, flops_per_rank: float, ms: float) -> float:
    """Whole-job throughput: every rank transforms its own replica (weak
    scaling), timed by the slowest rank."""
    return world * flops_per_rank / (ms * 1e-3) / 1e9


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle (test infrastructure) on bounded samples
# ---------------------------------------------------------------------------
def oracle_sample_step(x, rows: int, threads: int):
    """One bounded sample of the 8192^2 transform on the oracle: `rows` full
    row transforms (length nx) and `rows` full column transforms (length ny),
    i.e. rows/ny of the whole 2D job.  Returns the flops that represents."""
    import oracle
    ny, nx = x.shape
    oracle.fft1d_batch(x[:rows], dir=-1, threads=threads)
    cols = np.ascontiguousarray(x[:, :rows].T)
    oracle.fft1d_batch(cols, dir=-1, threads=threads)
    return flops_2d(nx, ny) * rows / ny


def cpu_baseline(x, budget_s: float = 12.0):
    import oracle
    threads = oracle.max_threads()
    rows = 256
    t = time.perf_counter()
    fl = oracle_sample_step(x, rows, threads)
    dt = time.perf_counter() - t
    reps = max(1, min(20, int(budget_s / max(dt, 1e-3))))
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        oracle_sample_step(x, rows, threads)
        times.append(time.perf_counter() - t)
    med = statistics.median(times)
    return {"value": fl / med / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"{rows} row FFTs + {rows} column FFTs (length 8192, FP64 recursive radix-2) of the "
                      f"8192x8192 input = {rows}/8192 of one 2D transform; median of {reps}"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    x = synth.normal_complex((NY, NX), seed=SEED)
    import oracle
    threads = oracle.max_threads()
    rows = 64
    for _ in range(args.warmup):
        oracle_sample_step(x, rows, threads)
    times = []
    fl = 0.0
    for _ in range(args.steps):
        t = time.perf_counter()
        fl = oracle_sample_step(x, rows, threads)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = fl * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "fft2d_c2c_8192x8192_forward", "nx": NX, "ny": NY, "batch": 1,
                       "inputs": "re/im N(0,1), seed 2506",
                       "sample_per_step": f"{rows} rows + {rows} columns of the 2D transform"},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": f"{rows} row + {rows} column FFTs of length 8192 per step"},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# This library
# ---------------------------------------------------------------------------
def time_plan(torch, plan, x, out, steps, warmup, pass_events=False):
    """Mean ms per execute (CUDA events on the current stream); optionally the
    mean per-pass durations from events recorded between the passes."""
    for _ in range(warmup):
        plan.execute(x, out=out)
    torch.cuda.synchronize()
    evs = []
    if pass_events:
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        for trip in evs:
            for e in trip:
                e.record()
        torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(steps):
        if pass_events:
            plan.set_pass_events(*evs[k])
        plan.execute(x, out=out)
    b.record()
    torch.cuda.synchronize()
    if pass_events:
        plan.set_pass_events(None, None, None)
    ms = a.elapsed_time(b) / steps
    passes = None
    if pass_events:
        r = [t[0].elapsed_time(t[1]) for t in evs]
        c = [t[1].elapsed_time(t[2]) for t in evs]
        passes = (sum(r) / steps, sum(c) / steps)
    return ms, passes


def time_plan_flushed(torch, plan, x, out, steps, scratch):
    """Mean and median ms per execute with L2 cold: before each timed call a
    scratch buffer twice the size of L2 is written, outside the timed events."""
    plan.execute(x, out=out)
    torch.cuda.synchronize()
    ts = []
    for k in range(steps):
        scratch.fill_(float(k))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        plan.execute(x, out=out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sum(ts) / len(ts), statistics.median(ts)


def forms(torch, g, steps, warmup, dev):
    """Secondary measurements (rank 0, N=1 only): other sizes, inverse, the
    split tensor-core path, the differentiation form and the ragged batch."""
    import synth
    out = {}
    # 2 x the 129 MB L2, written before each L2-cold call of the sizes that fit L2
    scratch = torch.empty(2 * 129 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for n in (1024, 2048, 4096, 8192):
        x = torch.from_numpy(synth.normal_complex((n, n), seed=SEED)).to(dev)
        y = torch.empty_like(x)
        for inv in (False, True):
            plan = g.get_plan(n, n, 1, inv, "fp32", dev)
            ms, _ = time_plan(torch, plan, x, y, max(10, steps // 4), 3)
            entry = {"ms": ms, "GFLOP/s": flops_2d(n, n) / ms / 1e6,
                     "HBM_GB/s_algorithmic": 32.0 * n * n / ms / 1e6,
                     "note": "fits L2 (hot)" if n <= 2048 else "larger than L2"}
            if n <= 2048:
                cold, cold_med = time_plan_flushed(torch, plan, x, y, 20, scratch)
                entry.update({"ms_l2_flushed": cold, "ms_l2_flushed_median": cold_med,
                              "HBM_GB/s_algorithmic_l2_flushed": 32.0 * n * n / cold / 1e6})
            out[f"fp32_{'inv' if inv else 'fwd'}_{n}"] = entry
        del x, y
    del scratch
    # split-FP16 tensor-core form on the precision workloads (noise + 8
    # exponentials), beside the FP32 path; relative difference of the two
    # results (the error against FP64 comes from the parity tests)
    xe = torch.from_numpy(synth.exp_mix_2d(8192, 8192, seed=SEED)[0]).to(dev)
    ye = torch.empty_like(xe)
    ref = g.get_plan(8192, 8192, 1, False, "fp32", dev).execute(xe).clone()
    plan = g.get_plan(8192, 8192, 1, False, "split_tc", dev)
    ms, _ = time_plan(torch, plan, xe, ye, max(10, steps // 4), 3)
    diff = float(torch.linalg.vector_norm(ye - ref) / torch.linalg.vector_norm(ref))
    out["split_tc_fwd_8192"] = {"ms": ms, "GFLOP/s": flops_2d(8192, 8192) / ms / 1e6,
                                "HBM_GB/s_algorithmic": 32.0 * 8192 * 8192 / ms / 1e6,
                                "rel_l2_vs_fp32_path": diff}
    del xe, ye, ref
    x1 = torch.from_numpy(synth.exp_mix_1d(16384, 4096, seed=SEED)[0]).to(dev)
    y1 = torch.empty_like(x1)
    ref = g.get_plan(4096, 1, 16384, False, "fp32", dev).execute(x1).clone()
    plan = g.get_plan(4096, 1, 16384, False, "split_tc", dev)
    ms, _ = time_plan(torch, plan, x1, y1, max(10, steps // 4), 3)
    diff = float(torch.linalg.vector_norm(y1 - ref) / torch.linalg.vector_norm(ref))
    out["split_tc_1d_4096x16384"] = {"ms": ms, "GFLOP/s": flops_2d(4096, 1, 16384) / ms / 1e6,
                                     "HBM_GB/s_algorithmic": 16.0 * 4096 * 16384 / ms / 1e6,
                                     "rel_l2_vs_fp32_path": diff}
    del x1, y1, ref
    # batch of 16384 1D length-4096 signals (one pass)
    x = torch.from_numpy(synth.exp_mix_1d(16384, 4096, seed=SEED)[0]).to(dev)
    y = torch.empty_like(x)
    plan = g.get_plan(4096, 1, 16384, False, "fp32", dev)
    ms, _ = time_plan(torch, plan, x, y, max(10, steps // 4), 3)
    out["fp32_1d_4096x16384"] = {"ms": ms, "GFLOP/s": flops_2d(4096, 1, 16384) / ms / 1e6,
                                 "HBM_GB/s_algorithmic": 16.0 * 4096 * 16384 / ms / 1e6}
    del x, y
    out.update(fourstep_form(torch, g, steps, dev))
    out.update(any_size_form(torch, g, steps, dev))
    out.update(energy_form(torch, g, dev))
    out.update(ragged_form(torch, g, steps, dev))
    out.update(diff_form(torch, g, steps, dev))
    return out


def energy_form(torch, g, dev):
    """Energy per transform from the board's NVML energy counter (the
    paper's Table 3 metric: runtime, average power, joules per 2D FFT),
    for its 1024 x 1024 workload and for 8192 x 8192; >= 2 s of back-to-back
    transforms each, board idle power alongside."""
    import synth
    from paper_2506_15437_gb300.energy import EnergyMeter, NVMLError
    try:
        meter = EnergyMeter.for_torch_device(dev)
        out = {"energy_idle_board_w": meter.idle_power_w(1.0)}
        for n in (1024, 8192):
            x = torch.from_numpy(synth.normal_complex((n, n), seed=SEED)).to(dev)
            y = torch.empty_like(x)
            plan = g.get_plan(n, n, 1, False, "fp32", dev)
            for _ in range(3):
                plan.execute(x, out=y)
            r = meter.measure(lambda: plan.execute(x, out=y), torch.cuda.synchronize, flops_2d(n, n),
                              min_seconds=2.0)
            out[f"energy_fp32_fwd_{n}"] = r
            del x, y
        return out
    except (NVMLError, AttributeError) as e:
        return {"energy": {"unavailable": str(e)}}


def any_size_form(torch, g, steps, dev):
    """Sizes that are not powers of two.  13-smooth lengths take the
    mixed-radix kernel (one HBM pass per axis: 1000 x 1000 beside the
    paper's 1024 x 1024, 1920 x 1080, 16384 signals of 3000 points, 16384
    signals of 4095 = 3^2 5 7 13 points), or, longer than one CTA holds, its
    four-step form (two passes: 32 signals of 10^6 points); other lengths
    Bluestein over the power-of-two path (16384 signals of the prime 4093,
    padded to M = 8192).  GFLOP/s uses the nominal 5 N log2 N of the
    transform's own size; the HBM figure counts one read and one write per
    axis or pass."""
    import math
    import synth
    out = {}
    for nx, ny, b in ((1000, 1000, 1), (1920, 1080, 1), (3000, 1, 16384), (1_000_000, 1, 32), (4095, 1, 16384),
                      (4093, 1, 16384)):
        x = torch.from_numpy(synth.uniform_complex((b, ny, nx), seed=SEED)).to(dev)
        y = torch.empty_like(x)
        plan = g.get_plan(nx, ny, b, False, "fp32", dev)
        ms, _ = time_plan(torch, plan, x, y, max(10, steps // 4), 3)
        n = nx * ny
        d = plan.describe()
        axes = 2 if ny > 1 or d["x"]["mixed_fourstep"][0] else 1
        out[f"fp32_any_{nx}x{ny}x{b}"] = {
            "ms": ms, "GFLOP/s_nominal": 5.0 * n * math.log2(n) * b / ms / 1e6,
            "HBM_GB/s_algorithmic": 16.0 * axes * n * b / ms / 1e6,
            "mixed": [d["x"]["mixed"], d["y"]["mixed"]], "mixed_fourstep": d["x"]["mixed_fourstep"],
            "bluestein_m": [d["x"]["bluestein_m"], d["y"]["bluestein_m"]], "transposes": d["transposes"]}
        del x, y
    return out


def fourstep_form(torch, g, steps, dev):
    """Long 1D transforms beyond one CTA: 4 x 2^24 points (four-step, two HBM
    passes) and 1 x 2^26 (three passes: 4096-point columns, a 4-point middle
    pass carrying the twiddles, 4096-point rows), both 512 MiB of input.  The
    HBM figure counts the two-pass minimum, 32 B per point."""
    import synth
    out = {}
    for n, b in ((1 << 24, 4), (1 << 26, 1)):
        x = torch.from_numpy(synth.uniform_complex((b, n), seed=SEED)).to(dev)
        y = torch.empty_like(x)
        plan = g.get_plan(n, 1, b, False, "fp32", dev)
        ms, passes = time_plan(torch, plan, x, y, max(10, steps // 4), 3, pass_events=True)
        d = plan.describe()
        out[f"fp32_1d_fourstep_{n}x{b}"] = {
            "ms": ms, "GFLOP/s": flops_2d(n, 1, b) / ms / 1e6,
            "HBM_GB/s_algorithmic": 32.0 * n * b / ms / 1e6,
            "passes_ms": {"cols": passes[0], "rows_twiddled_transposed": passes[1]},
            "n1_x_n2": [d["fourstep"]["n1"], d["fourstep"]["n2"]], "middle": d["fourstep"]["m"],
            "kernels": [k for k in (d["cols"]["kernel"], d["fourstep"]["mid"], d["rows"]["kernel"]) if k]}
        del x, y
    return out


def diff_form(torch, g, steps, dev):
    """L = sum w * |FFT2(x)|^2 for x [8][2048][2048], w U[0,1): one step is the
    forward transform, the loss and the adjoint (gradient).  Fused (what
    weighted_power_loss runs): forward rows; one column pass that sums the
    loss and runs the adjoint's column half on w (.) X; the adjoint's rows
    scaled by the upstream gradient read on the device -- 52 B per point
    (16 + 8 + 4 + 8 + 16).  Unfused, beside it: forward transform, loss
    reduction over X and w, weighted adjoint -- 76 B per point."""
    import synth
    b, n = 8, 2048
    x = torch.from_numpy(synth.uniform_complex((b, n, n), seed=SEED)).to(dev)
    w = torch.from_numpy(synth.mask((b, n, n), seed=SEED + 1)).to(dev)
    plan = g.get_plan(n, n, b, False, "fp32", dev)
    X = torch.empty_like(x)
    G = torch.empty_like(x)
    upstream = torch.ones(1, dtype=torch.float32, device=dev)  # dOut/dL, read on the device

    def step_unfused():
        plan.execute(x, out=X)
        plan.weighted_power(X, w)
        plan.backward_weighted_dev(X, w, upstream, 2.0, out=G)

    def step_fused():
        plan.weighted_power_adjoint(x, w, X)
        plan.backward_rows_scaled(X, upstream, 2.0, out=G)

    fl = 2 * flops_2d(n, n, b)
    ms_u = time_fn(torch, step_unfused, max(10, steps // 4))
    out = {"ms_unfused": ms_u, "HBM_GB/s_algorithmic_unfused": 76.0 * b * n * n / ms_u / 1e6}
    if plan.weighted_power_adjoint_parts() > 0:
        ms = time_fn(torch, step_fused, max(10, steps // 4))
        out.update({"ms": ms, "form": "fused", "GFLOP/s_two_transforms": fl / ms / 1e6,
                    "HBM_GB/s_algorithmic": 52.0 * b * n * n / ms / 1e6})
    else:
        out.update({"ms": ms_u, "form": "unfused", "GFLOP/s_two_transforms": fl / ms_u / 1e6,
                    "HBM_GB/s_algorithmic": 76.0 * b * n * n / ms_u / 1e6})
    return {"diff_8x2048x2048": out}


def time_fn(torch, fn, steps, warmup=3):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def ragged_form(torch, g, steps, dev):
    """512 independent 2D FFTs, each axis log-uniform on 32..1024 (seed 2506):
    one persistent launch replayed from a CUDA graph, against one plain
    launch pair per instance."""
    import synth
    nx, ny, offs, packed = synth.ragged_batch(512, seed=SEED)
    plan = g.RaggedPlan(nx, ny)
    x = torch.from_numpy(packed).to(dev)
    y = torch.empty_like(x)
    fl = sum(flops_2d(int(a), int(b)) for a, b in zip(nx, ny))
    byts = ragged_algorithmic_bytes(nx, ny)
    ms_graph = time_fn(torch, lambda: plan.execute(x, out=y), max(10, steps // 4))
    ms_loop = time_fn(torch, lambda: plan.execute_loop(x, out=y), max(5, steps // 10))
    plan.close()
    peak, peak_kind, _ = read_peaks()
    gbs = byts / ms_graph / 1e6
    return {"ragged_512": {"ms_graph": ms_graph, "ms_loop": ms_loop, "GFLOP/s": fl / ms_graph / 1e6,
                           "GFLOP/s_loop": fl / ms_loop / 1e6, "speedup_vs_loop": ms_loop / ms_graph,
                           "points": int(packed.size), "algorithmic_bytes": byts,
                           "HBM_GB/s_algorithmic": gbs, "frac_of_peak": gbs / peak,
                           "peak": f"{peak:.1f} GB/s ({peak_kind})"}}


def ragged_algorithmic_bytes(nx, ny, fused_max=8192):
    """One read and one write of complex64 per point per HBM pass: instances
    of at most `fused_max` points fit one CTA's shared memory, so they are
    charged one pass (16 B per point), larger ones two passes (32 B per
    point).  The kernel fuses only instances up to its 4096-element work
    item, so for those between 4096 and 8192 points this is a lower bound."""
    total = 0
    for a, b in zip(nx, ny):
        n = int(a) * int(b)
        total += (16 if n <= fused_max else 32) * n
    return float(total)


def profile_form(torch, name, steps, warmup, dev):
    """One secondary workload alone (for ncu): plan, warm-up, `steps` runs."""
    from paper_2506_15437_gb300 import build as _build
    _build.build()
    import paper_2506_15437_gb300 as g
    import synth
    if name == "ragged":
        nx, ny, _, packed = synth.ragged_batch(512, seed=SEED)
        plan = g.RaggedPlan(nx, ny)
        x = torch.from_numpy(packed).to(dev)
        run = lambda: plan.execute(x)  # noqa: E731
    elif name == "diff":
        b, n = 8, 2048
        x = torch.from_numpy(synth.uniform_complex((b, n, n), seed=SEED)).to(dev)
        w = torch.from_numpy(synth.mask((b, n, n), seed=SEED + 1)).to(dev)
        plan = g.Plan(n, n, b)
        X = torch.empty_like(x)
        upstream = torch.ones(1, dtype=torch.float32, device=dev)
        run = lambda: (plan.execute(x, out=X), plan.weighted_power(X, w),  # noqa: E731
                       plan.backward_weighted_dev(X, w, upstream, 2.0))
    elif name == "diff_fused":
        # the same step with the loss and the adjoint's column half fused
        # into the forward's column pass
        b, n = 8, 2048
        x = torch.from_numpy(synth.uniform_complex((b, n, n), seed=SEED)).to(dev)
        w = torch.from_numpy(synth.mask((b, n, n), seed=SEED + 1)).to(dev)
        plan = g.Plan(n, n, b)
        Y = torch.empty_like(x)
        G = torch.empty_like(x)
        upstream = torch.ones(1, dtype=torch.float32, device=dev)
        run = lambda: (plan.weighted_power_adjoint(x, w, Y),  # noqa: E731
                       plan.backward_rows_scaled(Y, upstream, 2.0, out=G))
    elif name == "fp32_8192":
        # the headline transform alone (row pass, column pass)
        x = torch.from_numpy(synth.normal_complex((8192, 8192), seed=SEED)).to(dev)
        plan = g.Plan(8192, 8192, 1)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    elif name == "mixed_fourstep_1e6":
        # 32 signals of 10^6 = 1000 x 1000 points: mixed-radix four-step (two passes)
        x = torch.from_numpy(synth.uniform_complex((32, 1_000_000), seed=SEED)).to(dev)
        plan = g.Plan(1_000_000, 1, 32)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    elif name == "small_1024":
        # one 1024 x 1024 array: rows and columns in one cooperative launch
        x = torch.from_numpy(synth.normal_complex((1024, 1024), seed=SEED)).to(dev)
        plan = g.Plan(1024, 1024, 1)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    elif name in ("bluestein_1001", "bluestein_4095"):
        # 32768 signals of 1001 = 7 11 13 points (one-pass fused Bluestein
        # over M = 2048) or 8192 signals of 4095 = 3^2 5 7 13 (fused, two
        # passes over M = 8192), planned with the mixed-radix kernel
        # switched off: both lengths are 13-smooth, so by default they run
        # mixed radix
        n, b = (1001, 32768) if name == "bluestein_1001" else (4095, 8192)
        x = torch.from_numpy(synth.uniform_complex((b, n), seed=SEED)).to(dev)
        os.environ["GB300FFT_MIXED"] = "0"
        plan = g.Plan(n, 1, b)
        del os.environ["GB300FFT_MIXED"]
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    elif name == "mixed_4095":
        # 8192 signals of 4095 = 3^2 5 7 13 points: mixed radix 15, 3, 7, 13
        x = torch.from_numpy(synth.uniform_complex((8192, 4095), seed=SEED)).to(dev)
        plan = g.Plan(4095, 1, 8192)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    elif name == "transpose_2d":
        # 4096 x 4093 (4093 prime): the y axis runs between two tiled transposes
        x = torch.from_numpy(synth.uniform_complex((4093, 4096), seed=SEED)).to(dev)
        plan = g.Plan(4096, 4093, 1)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    elif name == "mixed_3000":
        # 8192 signals of 3000 = 2^3 3 5^3 points (mixed radix, 196 MB each way)
        x = torch.from_numpy(synth.uniform_complex((8192, 3000), seed=SEED)).to(dev)
        plan = g.Plan(3000, 1, 8192)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    elif name.startswith("fourstep"):
        n, b = (1 << 24, 4) if name == "fourstep_2p24" else (1 << 26, 1)
        x = torch.from_numpy(synth.uniform_complex((b, n), seed=SEED)).to(dev)
        plan = g.Plan(n, 1, b)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    else:
        if name == "split_tc_8192":
            x = synth.exp_mix_2d(8192, 8192, seed=SEED)[0]
            plan = g.Plan(8192, 8192, 1, precision="split_tc")
        else:
            x = synth.exp_mix_1d(16384, 4096, seed=SEED)[0]
            plan = g.Plan(4096, 1, 16384, precision="split_tc" if name == "split_tc_1d" else "fp32")
        x = torch.from_numpy(x).to(dev)
        y = torch.empty_like(x)
        run = lambda: plan.execute(x, out=y)  # noqa: E731
    for _ in range(warmup + steps):
        run()
    torch.cuda.synchronize()
    print(json.dumps({"profile_form": name, "steps": steps, "warmup": warmup,
                      "schedule": plan.describe() if hasattr(plan, "describe") else None}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-forms", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--eager", action="store_true", help="enqueue the timed steps one by one (no CUDA graph)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-form", default=None,
                    choices=["split_tc_8192", "split_tc_1d", "fp32_1d", "fp32_8192", "ragged", "diff", "diff_fused", "bluestein_1001", "small_1024",
                             "mixed_fourstep_1e6", "mixed_4095",
                             "fourstep_2p24", "fourstep_2p26", "mixed_3000", "bluestein_4095", "transpose_2d"],
                    help="run only this secondary workload for --steps steps (for profilers); prints its schedule, not a metric line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.profile_form:
        return profile_form(torch, args.profile_form, args.steps, args.warmup, dev)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    from paper_2506_15437_gb300 import build as _build
    if rank == 0 or not _build.up_to_date():
        _build.build()
    if pg:
        pg.barrier()
    import paper_2506_15437_gb300 as g
    import synth

    x_host = torch.from_numpy(synth.normal_complex((NY, NX), seed=SEED + rank)).pin_memory()
    x = x_host.to(dev)
    out = torch.empty_like(x)
    plan = g.Plan(NX, NY, 1, inverse=False, precision="fp32")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        plan.execute(x, out=out)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for trip in evs:
        for e in trip:
            e.record()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    # The K timed steps are captured once into a CUDA graph (each step: its
    # three pass events as event-record nodes, the row and column kernels)
    # and replayed as one launch, so a slow or busy host cannot starve the
    # GPU between steps; --eager enqueues them one by one instead.
    graph = None
    timing = "eager"
    if not args.eager:
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                for k in range(args.steps):
                    plan.set_pass_events(*evs[k])
                    plan.execute(x, out=out)
            plan.set_pass_events(None, None, None)
            graph.replay()  # untimed
            torch.cuda.synchronize()
            timing = "cuda_graph"
        except Exception as exc:  # capture refused: time eagerly
            plan.set_pass_events(None, None, None)
            torch.cuda.synchronize()
            graph = None
            timing = f"eager (graph capture failed: {type(exc).__name__})"
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    start.record()
    t_host = time.perf_counter()
    if graph is not None:
        graph.replay()
    else:
        for k in range(args.steps):
            plan.set_pass_events(*evs[k])
            plan.execute(x, out=out)
    end.record()
    host_ms = (time.perf_counter() - t_host) * 1e3 / args.steps  # enqueue time per step (diagnostic)
    torch.cuda.synchronize()
    clocks.mark()
    if pg:
        pg.barrier()
    plan.set_pass_events(None, None, None)
    del graph  # the replayed graph is not needed again
    ms = max_over_ranks(pg, start.elapsed_time(end) / args.steps, dev)
    status = plan.status()
    rows_ms = sum(t[0].elapsed_time(t[1]) for t in evs) / args.steps
    cols_ms = sum(t[1].elapsed_time(t[2]) for t in evs) / args.steps
    time.sleep(0.25)
    clocks.stop()
    clk = clocks.summary()

    value = job_gflops(world, flops_2d(NX, NY), ms)

    # end to end through the public API with host buffers (fft_execute_host):
    # every step copies its pinned host input to the device, transforms it and
    # copies the result back to pinned host memory, all inside the timed
    # region; the library overlaps one step's upload with the previous
    # step's download
    out_host = torch.empty_like(x_host).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):
        plan.execute_host(x_host, out_host, device=dev)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(e2e_steps):
        plan.execute_host(x_host, out_host, device=dev)
    b.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(pg, a.elapsed_time(b) / e2e_steps, dev)
    nbytes = NX * NY * 8

    peak, peak_kind, _ = read_peaks()
    sched = plan.describe()
    dom_name, dom_ms = ((sched["rows"]["kernel"], rows_ms) if rows_ms >= cols_ms
                        else (sched["cols"]["kernel"], cols_ms))
    achieved = 16.0 * NX * NY / (dom_ms * 1e-3) / 1e9
    traffic = read_traffic(dom_name)
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "traffic": traffic, "algorithmic_bytes_per_launch": 16 * NX * NY,
                "passes_ms": {"rows": rows_ms, "cols": cols_ms}, "schedule": sched,
                "whole_step_frac": (32.0 * NX * NY / (ms * 1e-3) / 1e9) / peak}

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "fft2d_c2c_8192x8192_forward", "nx": NX, "ny": NY, "batch": 1,
                       "precision": "fp32", "inputs": "re/im N(0,1), seed 2506 (+rank)",
                       "l2": "inputs and outputs 512 MiB each, larger than L2; no flush"},
            "roofline": roofline,
            "e2e": {"value": job_gflops(world, flops_2d(NX, NY), e2e_ms), "unit": "GFLOP/s",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": 2 * args.steps,
            "clocks": clk, "status": status, "timing": timing,
            "host_enqueue_ms_per_step": host_ms}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(x_host.numpy())
    if rank == 0 and world == 1 and not args.no_forms:
        line["forms"] = forms(torch, g, args.steps, args.warmup, dev)
    if rank == 0:
        print(json.dumps(line))
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
