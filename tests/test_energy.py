"""Host logic of the NVML energy meter, against a stand-in NVML (no GPU)."""
import pytest

from paper_2506_15437_gb300.energy import EnergyMeter, NVMLError


class FakeNVML:
    """Two devices; the energy counter of each advances by `watts` per
    simulated second of the fake clock."""

    def __init__(self, watts=(100.0, 400.0)):
        self.watts = list(watts)
        self.t = 0.0
        self.uuids = ["GPU-aaaa-0001", "GPU-bbbb-0002"]

    def device_count(self):
        return len(self.uuids)

    def handle(self, i):
        if not 0 <= i < len(self.uuids):
            raise NVMLError("bad index")
        return i

    def uuid(self, h):
        return self.uuids[h]

    def energy_mj(self, h):
        return int(round(1_000_000 + self.watts[h] * self.t * 1000.0))

    def power_mw(self, h):
        return int(self.watts[h] * 1000)

    # fake time
    def clock(self):
        return self.t

    def advance(self, dt):
        self.t += dt


def test_selects_device_by_uuid_with_or_without_prefix():
    nv = FakeNVML()
    assert EnergyMeter(uuid="bbbb-0002", nvml=nv).h == 1
    assert EnergyMeter(uuid="GPU-AAAA-0001", nvml=nv).h == 0
    with pytest.raises(NVMLError):
        EnergyMeter(uuid="cccc", nvml=nv)


def test_measure_energy_per_transform_and_power():
    nv = FakeNVML()
    m = EnergyMeter(uuid="bbbb-0002", nvml=nv)
    calls = []

    def step():
        calls.append(1)
        nv.advance(0.001)  # 1 ms per transform

    r = m.measure(step, sync=lambda: None, flop_per_step=1e9, min_seconds=0.5, clock=nv.clock)
    assert r["steps"] == len(calls) >= 500
    assert r["seconds"] == pytest.approx(r["steps"] * 0.001)
    assert r["avg_power_w"] == pytest.approx(400.0, rel=1e-3)
    assert r["j_per_transform"] == pytest.approx(0.4, rel=1e-3)  # 400 W x 1 ms
    assert r["ms_per_transform"] == pytest.approx(1.0)
    assert r["gflop_per_j"] == pytest.approx(1.0 / 0.4, rel=1e-3)


def test_measure_stops_at_max_steps():
    nv = FakeNVML()
    m = EnergyMeter(index=0, nvml=nv)

    def step():
        nv.advance(1e-6)

    r = m.measure(step, sync=lambda: None, flop_per_step=1.0, min_seconds=10.0, clock=nv.clock, max_steps=1000)
    assert r["steps"] == 1000


def test_counter_that_does_not_advance_is_an_error():
    nv = FakeNVML(watts=(0.0, 0.0))
    m = EnergyMeter(index=0, nvml=nv)
    with pytest.raises(NVMLError):
        m.measure(lambda: nv.advance(0.01), sync=lambda: None, flop_per_step=1.0, min_seconds=0.05,
                  clock=nv.clock)


def test_idle_power():
    nv = FakeNVML()
    m = EnergyMeter(index=0, nvml=nv)
    assert m.idle_power_w(seconds=2.0, clock=nv.clock, sleep=nv.advance) == pytest.approx(100.0, rel=1e-3)
    assert m.power_w() == 100.0


def test_missing_library_raises_nvml_error():
    from paper_2506_15437_gb300.energy import _NVML
    with pytest.raises(NVMLError):
        _NVML(path="libdoes-not-exist.so.1")
