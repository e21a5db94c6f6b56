"""Host-side logic of bench.py (no GPU): the per-class rooflines and the
nvidia-smi fallback of the clock sampler."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1302_1861_b300 import inputs  # noqa: E402


def test_rooflines_per_step_arithmetic():
    w = inputs.config2(n_histories=1000)
    steps, per_rank = 2, 100_000_000
    # one step: 1 ms of onesweep, 2 ms of source, 10 ms of electrons
    prof = {"onesweep": (2.0, 8), "source": (4.0, 12), "electron": (20.0, 18), "band_sort": (2.0, 18),
            "photon": (0.0, 0)}
    counts = np.zeros(12)
    counts[6] = 3.0e8                                   # electron steps per step
    r = bench.rooflines_per_step(prof, steps, w, per_rank, {"hbm_gbs": 6000.0}, counts)
    assert set(r) == {"onesweep", "source", "electron"}  # no bytes for the band sort, no photon launches
    n = w.records.n
    assert abs(r["onesweep"]["achieved"] - 2 * n * 16 / 1e-3 / 1e9) < 1e-6   # 2 digit passes of 16 B
    assert abs(r["source"]["achieved"] - per_rank * 80 / 2e-3 / 1e9) < 1e-6
    assert abs(r["source"]["frac"] - r["source"]["achieved"] / 6000.0) < 1e-12
    e = r["electron"]
    assert abs(e["achieved"] - 3.0e8 / 1e-2 / 1e9) < 1e-9
    assert abs(e["peak"] - bench.THREAD_INST_PEAK / bench.THREAD_INST_PER_ELECTRON_STEP / 1e9) < 1e-9


def test_clock_sampler_parses_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    c.lines = ["0, 1980, 2032, 900.1, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2032, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2010, 2032, 940.0, 0x0, Not Active, Active, Not Active, Not Active",
               "garbage"]
    out = c.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2010.0 and out["sm_min_mhz"] == 1980.0
    assert out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
