"""Clock sampling of bench.py on the host, against a fake NVML (no GPU, nothing is changed)."""
import sys
import time
import types

import bench


def _fake_nvml(bits, sm=1965, mx=2032):
    m = types.ModuleType("pynvml")
    m.NVML_CLOCK_SM = 1
    calls = {"init": 0}

    def init():
        calls["init"] += 1

    def by_index(i):
        return ("gpu", i)

    def by_bus(_):
        raise RuntimeError("no bus ids here")

    m.nvmlInit = init
    m.nvmlDeviceGetHandleByIndex = by_index
    m.nvmlDeviceGetHandleByPciBusId = by_bus
    m.nvmlDeviceGetClockInfo = lambda h, kind: sm
    m.nvmlDeviceGetMaxClockInfo = lambda h, kind: mx
    m.nvmlDeviceGetCurrentClocksEventReasons = lambda h: bits
    return m, calls


def test_summary_median_max_and_reason_union():
    s = bench.clocks_summary([(2032.0, 2032.0, set()), (1900.0, 2032.0, {"sw_power_cap"}),
                              (2000.0, 2032.0, set())], "nvml")
    assert s["sm_mhz"] == 2000.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    e = bench.clocks_summary([], "nvml")
    assert e["reasons"] == ["unsampled"] and e["sm_mhz"] is None


def test_nvml_sampler_maps_reason_bits(monkeypatch):
    # sw_power_cap (0x4) and hw_thermal_slowdown (0x40) active; idle (0x1) is not reported
    fake, calls = _fake_nvml(0x4 | 0x40 | 0x1)
    monkeypatch.setitem(sys.modules, "pynvml", fake)
    with bench.Clocks(0) as c:
        c.mark()
        time.sleep(0.02)
    s = c.summary()
    assert calls["init"] == 1
    assert s["source"] == "nvml" and s["samples"] >= 2
    assert s["sm_mhz"] == 1965.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_nvml_sampler_quiet_gpu(monkeypatch):
    fake, _ = _fake_nvml(0x0, sm=2032)
    monkeypatch.setitem(sys.modules, "pynvml", fake)
    with bench.Clocks(0) as c:
        c.mark()
    s = c.summary()
    assert s["reasons"] == [] and s["sm_mhz"] == 2032.0
