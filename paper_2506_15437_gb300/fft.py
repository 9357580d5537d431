"""Python API over the C ABI: plans, fft2 and the autograd Function.

PyTorch only provides device memory and streams here.  Every transform runs
in libgb300fft.so's kernels; the only thing this module does is pass tensor
pointers and the current stream through ctypes.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _native as N

_PREC = {"fp32": N.FFT_PREC_FP32, "split_tc": N.FFT_PREC_SPLIT_FP16_TC,
         "split_fp16_tc": N.FFT_PREC_SPLIT_FP16_TC}


def _stream_handle(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _check_tensor(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Plan:
    """A dense plan: ``batch`` transforms of size ``[ny][nx]``."""

    def __init__(self, nx: int, ny: int, batch: int = 1, inverse: bool = False,
                 precision: str = "fp32"):
        lib = N.load()
        self.nx, self.ny, self.batch = int(nx), int(ny), int(batch)
        self.dir = N.FFT_INVERSE if inverse else N.FFT_FORWARD
        self.precision = precision
        self._lib = lib
        self._p = lib.fft_plan_create(self.nx, self.ny, self.batch, self.dir, _PREC[precision])
        if not self._p:
            raise N.FFTError(lib.fft_last_error(), f"fft_plan_create({nx}, {ny}, {batch})")

    @property
    def numel(self) -> int:
        return self.nx * self.ny * self.batch

    def _io(self, x, out):
        _check_tensor(x, torch.complex64, "input")
        if x.numel() != self.numel:
            raise ValueError(f"input has {x.numel()} elements, plan expects {self.numel}")
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_tensor(out, torch.complex64, "out")
            if out.numel() != self.numel:
                raise ValueError("out has the wrong size")
        return out

    def execute(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self._io(x, out)
        N.check(self._lib.fft_execute(self._p, x.data_ptr(), out.data_ptr(),
                                      _stream_handle(x.device)), "fft_execute")
        return out

    def execute_host(self, x: torch.Tensor, out: torch.Tensor | None = None, device=None) -> torch.Tensor:
        """The transform of a host (CPU) complex64 tensor into a host tensor,
        through the plan's device staging buffers (fft_execute_host).  Pinned
        tensors keep the copies asynchronous; successive calls overlap one
        call's upload with the previous call's download.  Ordered on the
        current stream of `device` (default: the current CUDA device)."""
        if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != torch.complex64 or not x.is_contiguous():
            raise ValueError("execute_host takes a contiguous complex64 CPU tensor")
        if x.numel() != self.numel:
            raise ValueError(f"input has {x.numel()} elements, plan expects {self.numel}")
        if out is None:
            out = torch.empty_like(x, pin_memory=x.is_pinned())
        elif out.is_cuda or out.dtype != torch.complex64 or not out.is_contiguous() or out.numel() != self.numel:
            raise ValueError("out must be a contiguous complex64 CPU tensor of the plan's size")
        dev = torch.device("cuda") if device is None else torch.device(device)
        N.check(self._lib.fft_execute_host(self._p, x.data_ptr(), out.data_ptr(), _stream_handle(dev)),
                "fft_execute_host")
        return out

    def backward(self, g: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self._io(g, out)
        N.check(self._lib.fft_backward(self._p, g.data_ptr(), out.data_ptr(),
                                       _stream_handle(g.device)), "fft_backward")
        return out

    def backward_weighted(self, X: torch.Tensor, w: torch.Tensor, scale: float,
                          out: torch.Tensor | None = None) -> torch.Tensor:
        out = self._io(X, out)
        _check_tensor(w, torch.float32, "w")
        if w.numel() != self.numel:
            raise ValueError("w has the wrong size")
        N.check(self._lib.fft_backward_weighted(self._p, X.data_ptr(), w.data_ptr(),
                                                ctypes.c_float(scale), out.data_ptr(),
                                                _stream_handle(X.device)),
                "fft_backward_weighted")
        return out

    def backward_weighted_dev(self, X: torch.Tensor, w: torch.Tensor, scale_dev: torch.Tensor,
                              scale: float = 1.0, out: torch.Tensor | None = None) -> torch.Tensor:
        """F^H (scale * scale_dev * w (.) X) with scale_dev a one-element
        float32 CUDA tensor read on the device (no host synchronisation)."""
        out = self._io(X, out)
        _check_tensor(w, torch.float32, "w")
        _check_tensor(scale_dev, torch.float32, "scale_dev")
        if w.numel() != self.numel or scale_dev.numel() != 1:
            raise ValueError("w must have the plan's size and scale_dev one element")
        N.check(self._lib.fft_backward_weighted_dev(self._p, X.data_ptr(), w.data_ptr(), scale_dev.data_ptr(),
                                                    ctypes.c_float(scale), out.data_ptr(),
                                                    _stream_handle(X.device)),
                "fft_backward_weighted_dev")
        return out

    def weighted_power(self, X: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
        """sum w*|X|^2 as a float64 0-d tensor (partials reduced by torch)."""
        _check_tensor(X, torch.complex64, "X")
        _check_tensor(w, torch.float32, "w")
        parts = self._lib.fft_weighted_power_parts(self._p)
        partials = torch.empty(parts, dtype=torch.float32, device=X.device)
        N.check(self._lib.fft_weighted_power(self._p, X.data_ptr(), w.data_ptr(),
                                             partials.data_ptr(), _stream_handle(X.device)),
                "fft_weighted_power")
        return partials.double().sum()

    def weighted_power_adjoint_parts(self) -> int:
        """Partials of the fused differentiation form, or 0 where the plan
        does not cover it (fft_weighted_power_adjoint_parts)."""
        n = self._lib.fft_weighted_power_adjoint_parts(self._p)
        return n if n > 0 else 0

    def weighted_power_adjoint(self, x: torch.Tensor, w: torch.Tensor, y: torch.Tensor | None = None):
        """(L, y): L = sum w*|F x|^2 as a float64 0-d tensor and y =
        F_cols^H (w (.) F x), the adjoint's column half, in two passes
        (fft_weighted_power_adjoint)."""
        y = self._io(x, y)
        _check_tensor(w, torch.float32, "w")
        if w.numel() != self.numel:
            raise ValueError("w has the wrong size")
        parts = self.weighted_power_adjoint_parts()
        if parts == 0:
            raise N.FFTError(N.FFT_ERR_UNSUPPORTED, "fft_weighted_power_adjoint")
        partials = torch.empty(parts, dtype=torch.float32, device=x.device)
        N.check(self._lib.fft_weighted_power_adjoint(self._p, x.data_ptr(), w.data_ptr(), partials.data_ptr(),
                                                     y.data_ptr(), _stream_handle(x.device)),
                "fft_weighted_power_adjoint")
        return partials.double().sum(), y

    def backward_rows_scaled(self, y: torch.Tensor, scale_dev: torch.Tensor | None = None, scale: float = 1.0,
                             out: torch.Tensor | None = None) -> torch.Tensor:
        """scale * scale_dev * F_rows^H y (fft_backward_rows_scaled); scale_dev
        a one-element float32 CUDA tensor read on the device, or None."""
        out = self._io(y, out)
        if scale_dev is not None:
            _check_tensor(scale_dev, torch.float32, "scale_dev")
            if scale_dev.numel() != 1:
                raise ValueError("scale_dev must have one element")
        N.check(self._lib.fft_backward_rows_scaled(self._p, y.data_ptr(),
                                                   None if scale_dev is None else scale_dev.data_ptr(),
                                                   ctypes.c_float(scale), out.data_ptr(), _stream_handle(y.device)),
                "fft_backward_rows_scaled")
        return out

    def set_pass_events(self, start=None, mid=None, end=None):
        """Record torch.cuda.Event objects around the row and column passes of
        every following execute/backward (None, None, None turns it off)."""
        h = [None if e is None else ctypes.c_void_p(e.cuda_event) for e in (start, mid, end)]
        N.check(self._lib.fft_plan_set_pass_events(self._p, *h), "fft_plan_set_pass_events")

    def status(self) -> int:
        return self._lib.fft_plan_status(self._p, _stream_handle(torch.device("cuda")))

    def autotune(self):
        """Time the candidate schedules and keep the fastest (cached on disk)."""
        N.check(self._lib.fft_plan_autotune(self._p, _stream_handle(torch.device("cuda"))), "fft_plan_autotune")

    def describe(self) -> dict:
        """The schedule this plan runs (kernels, elements per thread, tiles)."""
        import json
        buf = ctypes.create_string_buffer(2048)
        self._lib.fft_plan_describe(self._p, buf, 2048)
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_p", None):
            self._lib.fft_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ColumnPlan(Plan):
    """Only the column FFTs (length ny, down each column) of ``batch``
    [ny][nx] slices: the local step of a slab-decomposed 2D transform after
    its exchange (fft_plan_create_columns)."""

    def __init__(self, nx: int, ny: int, batch: int = 1, inverse: bool = False):
        lib = N.load()
        self.nx, self.ny, self.batch = int(nx), int(ny), int(batch)
        self.dir = N.FFT_INVERSE if inverse else N.FFT_FORWARD
        self.precision = "fp32"
        self._lib = lib
        self._p = lib.fft_plan_create_columns(self.nx, self.ny, self.batch, self.dir, N.FFT_PREC_FP32)
        if not self._p:
            raise N.FFTError(lib.fft_last_error(), f"fft_plan_create_columns({nx}, {ny}, {batch})")


def slab_pack(x: torch.Tensor, parts: int, batch: int, rows: int, nx: int, out: torch.Tensor | None = None):
    """out[s][b][y][x'] = x[b][y][s*w + x'] (w = nx/parts): the all-to-all
    chunk for each rank s, contiguous (fft_slab_pack)."""
    _check_tensor(x, torch.complex64, "x")
    if x.numel() != batch * rows * nx:
        raise ValueError("x must hold batch*rows*nx elements")
    out = torch.empty(parts, batch, rows, nx // parts, dtype=x.dtype, device=x.device) if out is None else out
    _check_tensor(out, torch.complex64, "out")
    N.check(N.load().fft_slab_pack(x.data_ptr(), out.data_ptr(), parts, batch, rows, nx, _stream_handle(x.device)),
            "fft_slab_pack")
    return out


def slab_unpack(x: torch.Tensor, parts: int, batch: int, rows: int, w: int, out: torch.Tensor | None = None):
    """out[b][r*rows + y][x'] = x[r][b][y][x']: the chunks received from every
    rank assembled into this rank's column slab (fft_slab_unpack)."""
    _check_tensor(x, torch.complex64, "x")
    if x.numel() != parts * batch * rows * w:
        raise ValueError("x must hold parts*batch*rows*w elements")
    out = torch.empty(batch, parts * rows, w, dtype=x.dtype, device=x.device) if out is None else out
    _check_tensor(out, torch.complex64, "out")
    N.check(N.load().fft_slab_unpack(x.data_ptr(), out.data_ptr(), parts, batch, rows, w, _stream_handle(x.device)),
            "fft_slab_unpack")
    return out


_cache: dict = {}
_cache_lock = threading.Lock()


def get_plan(nx: int, ny: int, batch: int, inverse: bool, precision: str, device) -> Plan:
    key = (nx, ny, batch, inverse, precision, torch.device(device).index)
    with _cache_lock:
        p = _cache.get(key)
        if p is None:
            with torch.cuda.device(device):
                p = Plan(nx, ny, batch, inverse, precision)
            _cache[key] = p
        return p


def _shape(x: torch.Tensor):
    if x.dim() < 2:
        raise ValueError("fft2 needs at least 2 dimensions ([..., ny, nx])")
    ny, nx = x.shape[-2], x.shape[-1]
    return nx, ny, max(1, x.numel() // max(1, nx * ny))


class FFT2Function(torch.autograd.Function):
    """Differentiable 2D transform: forward = fft_execute, backward = fft_backward
    (the conjugate-transpose transform, PyTorch's conjugate-Wirtinger VJP)."""

    @staticmethod
    def forward(ctx, x, inverse: bool = False, precision: str = "fp32"):
        x = x.contiguous()
        nx, ny, batch = _shape(x)
        plan = get_plan(nx, ny, batch, inverse, precision, x.device)
        ctx.plan = plan
        return plan.execute(x)

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.backward(grad.contiguous()), None, None


def fft2(x: torch.Tensor, inverse: bool = False, precision: str = "fp32") -> torch.Tensor:
    """Unnormalised 2D DFT over the last two axes of a complex64 CUDA tensor."""
    return FFT2Function.apply(x, inverse, precision)


class FFT1Function(torch.autograd.Function):
    """Differentiable 1D transform along the last axis.  Lengths up to 8192
    run in one pass; longer ones (up to 2^26) as the two-pass four-step
    decomposition.  backward = fft_backward, the conjugate transpose."""

    @staticmethod
    def forward(ctx, x, inverse: bool = False):
        x = x.contiguous()
        n = x.shape[-1]
        plan = get_plan(n, 1, max(1, x.numel() // max(1, n)), inverse, "fp32", x.device)
        ctx.plan = plan
        return plan.execute(x)

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.backward(grad.contiguous()), None


def fft1(x: torch.Tensor, inverse: bool = False) -> torch.Tensor:
    """Unnormalised 1D DFT along the last axis of a complex64 CUDA tensor."""
    if x.dim() < 1:
        raise ValueError("fft1 needs at least 1 dimension")
    return FFT1Function.apply(x, inverse)


class WeightedPowerLoss(torch.autograd.Function):
    """L = sum w * |FFT2(x)|^2 with a fused adjoint: dL/dx = 2 F^H (w (.) F x).
    Where the plan covers it, the forward's column pass also sums the loss
    and runs the adjoint's column half (fft_weighted_power_adjoint), so the
    backward is one scaled row pass (fft_backward_rows_scaled) and X = F x is
    never stored; otherwise the forward stores X and the weighting is folded
    into the adjoint's first pass (fft_backward_weighted_dev)."""

    @staticmethod
    def forward(ctx, x, w, precision: str = "fp32"):
        x = x.contiguous()
        w = w.contiguous()
        nx, ny, batch = _shape(x)
        plan = get_plan(nx, ny, batch, False, precision, x.device)
        ctx.plan = plan
        if plan.weighted_power_adjoint_parts() > 0:
            L, y = plan.weighted_power_adjoint(x, w)
            ctx.fused = True
            ctx.save_for_backward(y)
            return L.to(torch.float32)
        X = plan.execute(x)
        ctx.fused = False
        ctx.save_for_backward(X, w)
        return plan.weighted_power(X, w).to(torch.float32)

    @staticmethod
    def backward(ctx, gL):
        saved = ctx.saved_tensors
        # the upstream gradient stays on the device: the backward's pass
        # reads it, so backward issues no host synchronisation
        g = gL.detach().to(device=saved[0].device, dtype=torch.float32).reshape(1).contiguous()
        if ctx.fused:
            return ctx.plan.backward_rows_scaled(saved[0], g, 2.0), None, None
        X, w = saved
        return ctx.plan.backward_weighted_dev(X, w, g, 2.0), None, None


def weighted_power_loss(x: torch.Tensor, w: torch.Tensor, precision: str = "fp32") -> torch.Tensor:
    return WeightedPowerLoss.apply(x, w, precision)


def reorder_map(n: int, axis: int = 0, device="cuda") -> torch.Tensor:
    """Output position of each input index under the kernels' data movement
    alone (identity butterflies): the fused digit reversal."""
    lib = N.load()
    m = torch.empty(n, dtype=torch.int32, device=device)
    N.check(lib.fft_debug_reorder_map(n, axis, m.data_ptr(), _stream_handle(m.device)),
            "fft_debug_reorder_map")
    return m


def radices(n: int, axis: int = 0) -> list:
    lib = N.load()
    buf = (ctypes.c_int * 16)()
    k = lib.fft_debug_radices(n, axis, buf)
    if k < 0:
        raise N.FFTError(k, "fft_debug_radices")
    return [buf[i] for i in range(k)]


class RaggedPlan:
    """Many independent 2D transforms of mixed sizes (each axis a power of two
    in 32..1024), packed back to back, run as one persistent launch from a
    captured CUDA graph (fft_execute_ragged)."""

    def __init__(self, nx, ny, inverse: bool = False, precision: str = "fp32"):
        lib = N.load()
        self._lib = lib
        nx = [int(v) for v in nx]
        ny = [int(v) for v in ny]
        if len(nx) != len(ny):
            raise ValueError("nx and ny must have the same length")
        self.nx, self.ny = nx, ny
        self.count = len(nx)
        ax = (ctypes.c_int * self.count)(*nx)
        ay = (ctypes.c_int * self.count)(*ny)
        self.dir = N.FFT_INVERSE if inverse else N.FFT_FORWARD
        self._p = lib.fft_plan_create_ragged(self.count, ax, ay, self.dir, _PREC[precision])
        if not self._p:
            raise N.FFTError(lib.fft_last_error(), "fft_plan_create_ragged")

    def offset(self, i: int) -> int:
        v = ctypes.c_longlong(0)
        N.check(self._lib.fft_ragged_offset(self._p, int(i), ctypes.byref(v)), "fft_ragged_offset")
        return int(v.value)

    @property
    def total(self) -> int:
        return self.offset(self.count)

    def _io(self, x, out):
        _check_tensor(x, torch.complex64, "input")
        if x.numel() != self.total:
            raise ValueError(f"packed input has {x.numel()} elements, plan expects {self.total}")
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_tensor(out, torch.complex64, "out")
            if out.numel() != self.total:
                raise ValueError("out has the wrong size")
        return out

    def execute(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self._io(x, out)
        N.check(self._lib.fft_execute_ragged(self._p, x.data_ptr(), out.data_ptr(),
                                             _stream_handle(x.device)), "fft_execute_ragged")
        return out

    def execute_loop(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """The same transforms as one plain launch pair per instance (baseline)."""
        out = self._io(x, out)
        N.check(self._lib.fft_execute_ragged_loop(self._p, x.data_ptr(), out.data_ptr(),
                                                  _stream_handle(x.device)), "fft_execute_ragged_loop")
        return out

    def status(self) -> int:
        return self._lib.fft_plan_status(self._p, _stream_handle(torch.device("cuda")))

    def close(self):
        if getattr(self, "_p", None):
            self._lib.fft_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
