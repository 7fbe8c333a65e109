"""Host logic of bench.py that needs no GPU: the clock sampler keeps the
samples stamped inside the timed region and reports throttle reasons; the
DRAM-traffic record is used only for the source it was taken on."""
import json
import os
import stat
import time

import pytest

import bench

FAKE_SMI = r'''#!/usr/bin/env python3
import datetime, sys, time
reason = "{reason}"
while True:
    t = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    cols = ["Not Active"] * 4
    if reason:
        cols[["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"].index(reason)] = "Active"
    print(f"{{t}}, 0, {{1965}}, 2070, 900.0, 0x0, " + ", ".join(cols), flush=True)
    time.sleep(0.02)
'''


def _fake_smi(tmp_path, monkeypatch, reason=""):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(FAKE_SMI.format(reason=reason))
    f.chmod(f.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{d}{os.pathsep}{os.environ['PATH']}")


def test_clocks_keep_the_timed_region(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    c = bench.Clocks(0)
    time.sleep(0.1)  # samples before the region are dropped
    c.mark(0)
    time.sleep(0.25)
    c.mark(1)
    time.sleep(0.1)
    r = c.stop()
    assert r is not None
    assert r["sm_mhz"] == 1965.0 and r["sm_max_mhz"] == 2070.0 and r["reasons"] == []
    assert r["samples"] == r["samples_in_region"] >= 3
    # fewer samples than were written over the whole 0.45 s
    assert r["samples"] < 0.45 / 0.02


def test_clocks_short_region_takes_the_nearest_sample(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    c = bench.Clocks(0)
    c.mark(0)
    c.mark(1)
    time.sleep(0.1)
    r = c.stop()
    assert r["samples"] == 1 and r["samples_in_region"] == 0


@pytest.mark.parametrize("reason", ["hw_slowdown", "sw_power_cap"])
def test_clocks_report_throttle_reasons(tmp_path, monkeypatch, reason):
    _fake_smi(tmp_path, monkeypatch, reason)
    c = bench.Clocks(0)
    c.mark(0)
    time.sleep(0.1)
    c.mark(1)
    assert c.stop()["reasons"] == [reason]


def test_clocks_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.Clocks(0)
    c.mark(0)
    c.mark(1)
    assert c.stop() is None


def test_traffic_record_follows_the_source(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    cs = root / "paper_2301_04698_gb300" / "csrc"
    cs.mkdir(parents=True)
    (cs / "k.cu").write_text("// kernel\n")
    (cs / "other.cu").write_text("// another kernel\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.src_hash(["k.cu"])
    rec = {"cg_wave": {"files": ["k.cu"], "src": h, "per": "cell-iteration", "dram_bytes_per_unit": 25.0}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.traffic_for("cg_wave", 1000) == 25000.0
    assert bench.traffic_for("scalar", 1000) is None
    (cs / "other.cu").write_text("// another kernel, changed\n")   # not this kernel's source
    assert bench.traffic_for("cg_wave", 1000) == 25000.0
    (cs / "k.cu").write_text("// kernel, changed\n")
    assert bench.src_hash(["k.cu"]) != h
    assert bench.traffic_for("cg_wave", 1000) is None
