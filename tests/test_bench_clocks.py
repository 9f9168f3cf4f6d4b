"""Host logic of bench.py's clock record: the nvidia-smi sampler keeps the
samples taken inside the timed region (a fake nvidia-smi on PATH stands in for
the real one; no GPU is involved)."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

FAKE = r'''#!{python}
import os, sys, time
args = sys.argv[1:]
if "-lms" not in args:  # probe: accept the ids listed in FAKE_SMI_OK
    ok = os.environ.get("FAKE_SMI_OK", "0").split(",")
    if args[args.index("-i") + 1] in ok:
        print("0")
        sys.exit(0)
    sys.exit(6)
ms = int(args[args.index("-lms") + 1])
k = 0
while True:
    t = time.time()
    stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int((t % 1) * 1000)
    sm = 1100 if k == 0 else 2070
    slow = "Active" if k == 3 else "Not Active"
    print(f"{{stamp}}, 0, {{sm}}, 2070, 700.00, 0x0000000000000000, Not Active, Not Active, Not Active, {{slow}}",
          flush=True)
    k += 1
    time.sleep(ms / 1000.0)
'''


def _line(t, sm, power_cap="Not Active"):
    stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int((t % 1) * 1000)
    return f"{stamp}, 0, {sm}, 2070, 900.50, 0x0, Not Active, Not Active, Not Active, {power_cap}"


def test_parse_keeps_region_samples():
    c = bench.ClockSampler(0)
    t = time.time()
    c.t0, c.t1 = t, t + 0.5
    r = c.parse([_line(t - 0.3, 900), _line(t + 0.1, 2070), _line(t + 0.3, 2040, "Active"), _line(t + 0.9, 600)])
    assert r["samples_in_region"] == 2 and r["samples"] == 2
    assert r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_parse_short_region_takes_nearest_sample():
    c = bench.ClockSampler(0)
    t = time.time()
    c.t0, c.t1 = t, t + 0.05
    r = c.parse([_line(t - 0.3, 900), _line(t + 0.12, 2070), _line(t + 0.4, 1500)])
    assert r["samples_in_region"] == 0 and r["samples"] == 1 and r["sm_mhz"] == 2070.0


def test_parse_without_stamps_or_lines():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 0.0, 1.0
    r = c.parse(["garbage", "N/A, 0, 2070, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert r["samples"] == 1 and r["sm_mhz"] == 2070.0  # unparsable stamp: all samples
    assert c.parse([])["reasons"] == ["no samples"]


def test_sampler_with_fake_nvidia_smi(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    c = bench.ClockSampler(0, interval_ms=50)
    c.start()
    time.sleep(0.5)  # the first (idle) sample lies before the region, even with a slow interpreter start
    c.region_start()
    time.sleep(0.5)
    c.region_end()
    r = c.stop()
    assert r["samples_in_region"] >= 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0


def test_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


def _fake_smi(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(python=sys.executable))
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])


def test_smi_id_takes_the_first_accepted_id(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,GPU-0a1b")
    monkeypatch.setenv("FAKE_SMI_OK", "5,GPU-0a1b,0,1,2")
    assert bench.ClockSampler.smi_id(0) == "5" and bench.ClockSampler.smi_id(1) == "GPU-0a1b"
    assert bench.ClockSampler.smi_id(2) == "2"
    monkeypatch.setenv("FAKE_SMI_OK", "0")  # a container that shows its one GPU as index 0
    assert bench.ClockSampler.smi_id(0) == "0"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    monkeypatch.setenv("FAKE_SMI_OK", "1")
    assert bench.ClockSampler.smi_id(1) == "1"


def test_smi_id_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3")
    assert bench.ClockSampler.smi_id(0) == "0"
