"""Energy and energy-delay product of a GPU run (the paper's Sec. 7 objectives).

The paper reads node and GPU power from Cray counters through APEX; on this
GPU the same quantity comes from NVML's total-energy counter (millijoules
since the driver loaded), read before and after a run.  Nothing here changes
any GPU setting; it only reads a counter.

    with EnergyMeter(device=0) as m:
        run()
    m.joules, m.seconds, m.edp   # energy, wall time, energy x time
"""
from __future__ import annotations

import ctypes
import time


class _NvmlLib:
    """The four NVML calls the meter needs, through ctypes on the driver's
    libnvidia-ml (for machines without the pynvml module).  Read-only."""

    def __init__(self):
        self._l = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"NVML {what} failed with code {rc}")

    def nvmlInit(self):
        self._ok(self._l.nvmlInit_v2(), "init")

    def nvmlShutdown(self):
        self._ok(self._l.nvmlShutdown(), "shutdown")

    def nvmlDeviceGetHandleByIndex(self, i):
        h = ctypes.c_void_p()
        self._ok(self._l.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(i), ctypes.byref(h)), "device handle")
        return h

    def nvmlDeviceGetTotalEnergyConsumption(self, h):
        mj = ctypes.c_ulonglong()
        self._ok(self._l.nvmlDeviceGetTotalEnergyConsumption(h, ctypes.byref(mj)), "energy counter")
        return mj.value


class EnergyMeter:
    def __init__(self, device: int = 0, nvml=None):
        self.device = device
        self._nvml = nvml
        self.joules = None
        self.seconds = None

    def _lib(self):
        if self._nvml is None:
            try:
                import pynvml
                self._nvml = pynvml
            except ImportError:
                self._nvml = _NvmlLib()
        return self._nvml

    def __enter__(self):
        nv = self._lib()
        nv.nvmlInit()
        self._h = nv.nvmlDeviceGetHandleByIndex(self.device)
        self._sync()
        self._e0 = nv.nvmlDeviceGetTotalEnergyConsumption(self._h)
        self._t0 = time.perf_counter()
        return self

    def _sync(self):
        try:
            import torch
            if torch.cuda.is_available():
                torch.cuda.synchronize(self.device)
        except ImportError:
            pass

    def __exit__(self, *exc):
        nv = self._lib()
        self._sync()
        e1 = nv.nvmlDeviceGetTotalEnergyConsumption(self._h)
        self.seconds = time.perf_counter() - self._t0
        self.joules = (e1 - self._e0) / 1000.0
        nv.nvmlShutdown()
        return False

    @property
    def edp(self) -> float:
        return self.joules * self.seconds

    @property
    def watts(self) -> float:
        return self.joules / self.seconds if self.seconds else 0.0


def objective_value(metric: str, seconds: float, joules: float | None) -> float:
    """The quantity the tuner minimises: run time, energy or energy x time."""
    if metric == "time":
        return seconds
    if joules is None:
        raise ValueError("energy metrics need an energy reading")
    if metric == "energy":
        return joules
    if metric == "edp":
        return joules * seconds
    raise ValueError(f"unknown metric {metric}")
