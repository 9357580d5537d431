"""Energy per transform from the GPU's own energy counter (NVML).

The paper compares accelerator and CPU by runtime, average power and energy
per 2D transform (Section 5, Table 3: a 1024 x 1024 FFT).  This module gives
the GPU side of that comparison: it reads NVML's total-energy counter
(millijoules since the driver loaded) around a run of back-to-back
transforms, and reports joules per transform, average board power and
GFLOP/J.

Only reads: it never changes a clock, power limit or any other device
setting.  NVML is reached through ctypes (libnvidia-ml.so.1 ships with the
driver); a stand-in object with the same methods can be passed instead, which
is how the host logic is tested without a GPU.
"""
from __future__ import annotations

import ctypes
import time


class NVMLError(RuntimeError):
    pass


class _NVML:
    """The few NVML entry points used here, bound through ctypes."""

    def __init__(self, path: str = "libnvidia-ml.so.1"):
        try:
            self._lib = ctypes.CDLL(path)
        except OSError as e:
            raise NVMLError(f"NVML not available: {e}") from e
        self._check(self._lib.nvmlInit_v2(), "nvmlInit_v2")

    def _check(self, rc: int, what: str):
        if rc != 0:
            raise NVMLError(f"{what} failed (nvmlReturn {rc})")

    def device_count(self) -> int:
        n = ctypes.c_uint(0)
        self._check(self._lib.nvmlDeviceGetCount_v2(ctypes.byref(n)), "nvmlDeviceGetCount_v2")
        return n.value

    def handle(self, index: int):
        h = ctypes.c_void_p()
        self._check(self._lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)),
                    "nvmlDeviceGetHandleByIndex_v2")
        return h

    def uuid(self, h) -> str:
        buf = ctypes.create_string_buffer(96)
        self._check(self._lib.nvmlDeviceGetUUID(h, buf, ctypes.c_uint(96)), "nvmlDeviceGetUUID")
        return buf.value.decode()

    def energy_mj(self, h) -> int:
        e = ctypes.c_ulonglong(0)
        self._check(self._lib.nvmlDeviceGetTotalEnergyConsumption(h, ctypes.byref(e)),
                    "nvmlDeviceGetTotalEnergyConsumption")
        return e.value

    def power_mw(self, h) -> int:
        p = ctypes.c_uint(0)
        self._check(self._lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(p)), "nvmlDeviceGetPowerUsage")
        return p.value

    def shutdown(self):
        self._lib.nvmlShutdown()


def _norm_uuid(u: str) -> str:
    u = u.strip().lower()
    return u[4:] if u.startswith("gpu-") else u


class EnergyMeter:
    """Energy counter of one GPU.

    ``uuid`` selects the device (the CUDA device's UUID, with or without the
    ``GPU-`` prefix); without it NVML index ``index`` is used.  ``nvml`` may
    be a stand-in with ``device_count/handle/uuid/energy_mj/power_mw``.
    """

    def __init__(self, uuid: str | None = None, index: int = 0, nvml=None):
        self.nvml = nvml if nvml is not None else _NVML()
        if uuid is not None:
            want = _norm_uuid(uuid)
            for i in range(self.nvml.device_count()):
                h = self.nvml.handle(i)
                if _norm_uuid(self.nvml.uuid(h)) == want:
                    self.h = h
                    break
            else:
                raise NVMLError(f"no NVML device with UUID {uuid}")
        else:
            self.h = self.nvml.handle(index)

    @classmethod
    def for_torch_device(cls, device=None, nvml=None) -> "EnergyMeter":
        import torch
        props = torch.cuda.get_device_properties(device if device is not None else torch.cuda.current_device())
        return cls(uuid=str(props.uuid), nvml=nvml)

    def read_mj(self) -> int:
        return self.nvml.energy_mj(self.h)

    def power_w(self) -> float:
        return self.nvml.power_mw(self.h) / 1000.0

    def measure(self, step, sync, flop_per_step: float, min_seconds: float = 2.0,
                clock=time.perf_counter, max_steps: int = 1 << 22) -> dict:
        """Run ``step()`` back to back for at least ``min_seconds`` (``sync()``
        ends each batch of launches) and return the energy it took.

        The counter is read after a sync on both sides, so the interval holds
        only this work (and the board's idle draw, which the result includes,
        as the paper's per-run power figures do)."""
        sync()
        e0, t0 = self.read_mj(), clock()
        steps, batch = 0, 1
        while True:
            for _ in range(batch):
                step()
            steps += batch
            sync()
            el = clock() - t0
            if el >= min_seconds or steps >= max_steps:
                break
            # grow the batch so host checks stay rare
            batch = min(batch * 2, max_steps - steps)
        e1 = self.read_mj()
        joules = (e1 - e0) / 1000.0
        if joules <= 0 or el <= 0:
            raise NVMLError("energy counter did not advance over the run")
        return {"steps": steps, "seconds": el, "joules": joules,
                "avg_power_w": joules / el, "j_per_transform": joules / steps,
                "ms_per_transform": 1e3 * el / steps,
                "gflop_per_j": flop_per_step * steps / joules / 1e9}

    def idle_power_w(self, seconds: float = 1.0, clock=time.perf_counter, sleep=time.sleep) -> float:
        """Average board power over ``seconds`` with nothing launched."""
        e0, t0 = self.read_mj(), clock()
        sleep(seconds)
        e1, t1 = self.read_mj(), clock()
        return (e1 - e0) / 1000.0 / max(t1 - t0, 1e-9)
