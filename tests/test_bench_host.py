"""Host-side logic of bench.py, without a GPU: the algorithmic bytes behind
the roofline, the count of sort launches the JSON line claims, the summary
of the nvidia-smi clock samples, and the reference arm (the oracle on the
host cores) end to end."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2303_05599_gb300 import workloads as W  # noqa: E402


def test_algorithmic_bytes():
    # FP32 two-row: (24 link + 8 phi + 16 e + 8 pi) floats read and written,
    # plus 48 site-field floats written
    assert bench.field_bytes_per_site(1) == 640
    assert bench.field_bytes_per_site(0) == (36 + 8 + 16 + 8) * 2 * 8 + 48 * 8 == 1472
    # a particle: 14 reals read and written plus its species index; a site:
    # 48 site-field reals and 8 scalar reals read
    assert bench.push_bytes(1, 1000, 64) == 116 * 1000 + 224 * 64
    assert bench.push_bytes(0, 1000, 64) == 228 * 1000 + 448 * 64


def test_leapfrog_and_site_field_bytes_are_itemised():
    # the leapfrog's own bytes (448 B per FP32 two-row site: every field read and written once) and
    # the 192 B site-field write add up to the fused launch's bytes
    assert bench.leapfrog_bytes_per_site(1) == 448
    assert bench.site_field_bytes_per_site(1) == 192
    assert bench.leapfrog_bytes_per_site(0) == 1088
    for prec in (0, 1):
        assert bench.field_bytes_per_site(prec) == (bench.leapfrog_bytes_per_site(prec)
                                                    + bench.site_field_bytes_per_site(prec))


def test_timed_window_ends_on_a_reunitarising_step():
    # step n re-unitarises when (n + 1) % every == 0
    for pre in (3, 13, 40, 63, 64, 100):
        for K in (1, 5, 20, 60, 64, 200):
            start = bench.timed_window_start(pre, K, 64)
            assert start >= pre
            assert any((n + 1) % 64 == 0 for n in range(start, start + K)), (pre, K, start)
            # not moved when the window already holds one
            if any((n + 1) % 64 == 0 for n in range(pre, pre + K)):
                assert start == pre
    assert bench.timed_window_start(13, 20, 64) == 44
    assert bench.timed_window_start(13, 20, 0) == 13


def test_representatives_weight_each_lattice_size():
    ws = W.config_batched_events()
    reps = bench.representatives(ws)
    assert [ws[i].N for i, _ in reps] == [64, 128, 256]
    assert [c for _, c in reps] == [22, 21, 21]
    assert sum(c for _, c in reps) == len(ws)


def test_sort_launches():
    # the default batch: two motion classes on 256^2 -> keys below 2^17, three
    # 8-bit passes: keys, 3 x (histogram, three scans, scatter), gather
    ws = [W.config_n256() for _ in range(30)]
    assert bench.sort_launches(ws) == 17
    # one motion class on 16^2: keys below 2^8, one pass
    w = W.Workload("one", N=16, L_fm=1.0, species=[W.Species(W.M_CHARM, 0.0, 10, W.REP_F, W.MOM_FIXED_PT, 0.5)])
    assert bench.sort_launches([w]) == 7
    # static quarks and eikonal partons are classes of their own
    w.species.append(W.Species(math.inf, 0.0, 10, W.REP_A, W.MOM_FIXED_PT, 0.0))
    w.species.append(W.Species(0.0, 0.0, 10, W.REP_F, 3, 10.0))
    assert bench.sort_launches([w]) == 12  # 3 x 256 - 1 needs 10 bits: two passes


def test_clock_summary():
    lines = ["0, 2070, 2070, 905.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
             "0, 2055, 2070, 910.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "0, 2070, 2070, 912.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "malformed line\n",
             "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n"]
    s = bench.ClockSampler.summarise(lines)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    slow = ["0, 1200, 2070, 700, 0x8, Active, Not Active, Active, Not Active\n"]
    assert bench.ClockSampler.summarise(slow)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarise([])["samples"] == 0


class _FakeNvml:
    """NVML read queries answered from fixed values (no GPU, no driver)."""

    def __init__(self, reasons):
        self.reasons = reasons
        self.bus = None

    def nvmlInit_v2(self):
        return 0

    def nvmlShutdown(self):
        return 0

    def nvmlDeviceGetHandleByPciBusId_v2(self, bus, handle):
        self.bus = bus.value
        handle._obj.value = 1234
        return 0

    def nvmlDeviceGetClockInfo(self, h, kind, out):
        assert kind == 1  # NVML_CLOCK_SM
        out._obj.value = 1980
        return 0

    def nvmlDeviceGetMaxClockInfo(self, h, kind, out):
        out._obj.value = 2070
        return 0

    def nvmlDeviceGetCurrentClocksThrottleReasons(self, h, out):
        out._obj.value = self.reasons
        return 0


def test_nvml_clock_sampler(monkeypatch):
    import time
    import types
    import torch
    fake = _FakeNvml(0x4 | 0x1)  # sw_power_cap, and GPU idle (not reported)
    monkeypatch.setattr(bench.ctypes, "CDLL", lambda name: fake)
    props = types.SimpleNamespace(pci_domain_id=0, pci_bus_id=0x1b, pci_device_id=0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: props)
    s = bench.NvmlClockSampler(0)
    assert s.start()
    time.sleep(0.05)
    rec = s.stop()
    assert fake.bus == b"00000000:1b:00.0"
    assert rec["samples"] >= 2 and rec["sm_mhz"] == 1980.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["source"] == "nvml"


def test_reference_arm_prints_one_line_without_a_gpu():
    # the reference arm times the oracle on the host cores: one JSON line with
    # the arm's metric and unit, no host-device bytes, and the oracle as its
    # CPU baseline (a few seconds of CPU work at one step)
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "site-updates/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["config"]["workload"] == "batched64"
