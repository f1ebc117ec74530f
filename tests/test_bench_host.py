"""CPU checks of the benchmark's host logic: the clock sampler's parsing of
nvidia-smi output (median clock, throttle reasons), the roofline peak's
source (the measured HBM bandwidth, else the stated fallback), and the flop
count per acoustic cell update."""
import json
import os
import stat
import time

import pytest

import bench


def _fake_smi(tmp_path, lines):
    """An executable `nvidia-smi` that records its arguments in args.txt,
    prints `lines` once, then idles."""
    script = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{ln}'" for ln in lines)
    script.write_text(f"#!/bin/sh\necho \"$@\" > {tmp_path}/args.txt\n{body}\nexec sleep 30\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_parses_clocks_and_reasons(tmp_path, monkeypatch):
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1950, 2070, 1350.2, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    ck = bench.ClockSampler("0")
    t0 = time.time()
    while time.time() - t0 < 10 and open(ck.f.name).read().count("\n") < len(lines):
        time.sleep(0.05)
    out = ck.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    out = bench.ClockSampler("0").stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_roofline_peak_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6788.3, "bf16_tflops": 1886.0}))
    assert bench.measured_peaks() == (6788.3, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("not json")
    assert bench.measured_peaks() == (6800.0, "fallback")


def test_flop_count_per_acoustic_cell_update():
    """3 components x 76 orbit-sum adds, 230 multiply-adds of the three nodes'
    two time combinations (2 flops each), 4 Simpson face sums x 3 components
    (a multiply-add and an add), 8 flux scalings, and per component two
    differences and two multiply-adds in the update."""
    assert bench.ACOUSTIC_FLOP_PER_CELL == 3 * 76 + 230 * 2 + 4 * 3 * 3 + 8 + 3 * (2 + 2 * 2) == 750


def test_clock_sampler_follows_a_remapped_device(tmp_path, monkeypatch):
    """Under CUDA_VISIBLE_DEVICES the process's CUDA device 1 is the host's
    GPU 5: without a UUID the sampler selects GPU 5, and with one it selects
    by UUID -- never the process-local index."""
    import types
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3,5")
    fake = types.SimpleNamespace(cuda=types.SimpleNamespace(
        get_device_properties=lambda d: types.SimpleNamespace(name="gpu")))
    monkeypatch.setitem(__import__("sys").modules, "torch", fake)
    assert bench.smi_device(1) == "5"
    fake.cuda.get_device_properties = lambda d: types.SimpleNamespace(uuid="1234abcd-0000-1111-2222-333344445555")
    assert bench.smi_device(1) == "GPU-1234abcd-0000-1111-2222-333344445555"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, ["5, 2070, 2070, 900.0, 0x0, Not Active, Not Active, "
                                                    "Not Active, Not Active"]) + os.pathsep + os.environ["PATH"])
    ck = bench.ClockSampler(bench.smi_device(1))
    t0 = time.time()
    while time.time() - t0 < 10 and not (tmp_path / "args.txt").exists():
        time.sleep(0.05)
    ck.stop()
    args = (tmp_path / "args.txt").read_text().split()
    assert args[:2] == ["-i", "GPU-1234abcd-0000-1111-2222-333344445555"]


def test_pareto_front_and_rate_at_equal_l1():
    """The equal-L1 comparison of the learned-tagging runs: a Pareto front
    keeps the points no other point beats (lower L1 and higher rate), and
    rate_at interpolates a front in log L1 / log rate, is None below its
    lowest L1 and holds its best rate beyond its largest."""
    import math
    pts = [(2e-3, 3.0), (1e-3, 1.0), (1.5e-3, 0.5), (3e-3, 2.0), (4e-3, 4.0)]
    assert bench.pareto_front(pts) == [(1e-3, 1.0), (2e-3, 3.0), (4e-3, 4.0)]
    fr = [(1e-3, 1.0), (4e-3, 4.0)]
    assert bench.rate_at(fr, 5e-4) is None
    assert math.isclose(bench.rate_at(fr, 2e-3), 2.0)
    assert math.isclose(bench.rate_at(fr, 1e-3), 1.0)
    assert bench.rate_at(fr, 1e-2) == 4.0
    assert bench.rate_at([], 1e-3) is None


def test_roofline_traffic_comes_from_the_committed_record(tmp_path):
    """roofline.traffic is the ncu record of the committed summary when it
    covers the timed tiling and the kernel's sources are unchanged (their
    hash); otherwise it is None with the reason."""
    t = {"tile": (32, 8), "threads": 128, "persistent": False}
    h = bench.kernel_source_hash()
    rec = tmp_path / "p.md"
    rec.write_text(f"x\ntraffic: tiling=32x8x128 bytes_per_launch=1951111424 source_hash={h}\n")
    assert bench.profiled_traffic(t, str(rec))[0] == 1951111424.0
    rec.write_text("traffic: tiling=32x8x128 bytes_per_launch=1951111424 source_hash=0000000000000000\n")
    v, why = bench.profiled_traffic(t, str(rec))
    assert v is None and why.startswith("stale")
    v, why = bench.profiled_traffic({"tile": (32, 16), "threads": 192, "persistent": False}, str(rec))
    assert v is None
    assert bench.profiled_traffic(t, str(tmp_path / "missing.md"))[0] is None
