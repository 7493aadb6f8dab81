"""Host checks of bench.py's clock record: samples are filtered by
nvidia-smi's own timestamp to the timed region, throttle reasons are read
per sample, and a region too short for any sample falls back to the whole
run and says so.  A fake nvidia-smi on PATH stands in for the real one."""
from __future__ import annotations

import os
import stat
import sys
import time

import pytest

import bench

FAKE = r'''#!{py}
import datetime, os, sys, time
until = float(os.environ["FAKE_CAP_UNTIL"])  # power cap active before this time
while True:
    now = datetime.datetime.now()
    cap = "Active" if time.time() < until else "Not Active"
    sm = 1500 if cap == "Active" else 2070
    print(now.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3] + ", 0, %d, 2070, 612.5, 0x0, Not Active, "
          "Not Active, Not Active, %s" % (sm, cap), flush=True)
    time.sleep(0.01)
'''


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.replace("{py}", sys.executable))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    return exe


def test_samples_inside_the_timed_region_only(fake_smi, monkeypatch):
    cap_until = time.time() + 0.1
    monkeypatch.setenv("FAKE_CAP_UNTIL", str(cap_until))
    s = bench.ClockSampler(0, period_ms=10)
    s.start()
    time.sleep(max(0.0, cap_until - time.time()) + 0.05)  # the power-capped samples
    s.begin()
    time.sleep(0.3)
    s.end()
    time.sleep(0.1)
    c = s.stop()
    assert c["window"] == "timed steps"
    assert c["samples"] >= 5
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == []


def test_reasons_seen_in_the_region_are_reported(fake_smi, monkeypatch):
    monkeypatch.setenv("FAKE_CAP_UNTIL", str(time.time() + 100.0))
    s = bench.ClockSampler(0, period_ms=10)
    s.begin()              # every sample of the region is power-capped
    s.start()
    time.sleep(0.4)
    s.end()
    c = s.stop()
    assert c["window"] == "timed steps"
    assert "sw_power_cap" in c["reasons"]


def test_short_region_falls_back_to_the_whole_run(fake_smi, monkeypatch):
    monkeypatch.setenv("FAKE_CAP_UNTIL", "0")
    s = bench.ClockSampler(0, period_ms=10)
    s.start()
    time.sleep(0.3)
    t = bench.datetime.datetime.now()
    s.region = [t, t - bench.datetime.timedelta(seconds=1)]  # empty region
    c = s.stop()
    assert c["window"].startswith("whole run")
    assert c["samples"] >= 3


def test_missing_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]


# A fake nvidia-smi that knows one GPU, physical index 3, by UUID or index.
FAKE_ID = r'''#!{py}
import sys
ids = [a.split("=", 1)[1] for a in sys.argv[1:] if a.startswith("--id=")]
if ids and ids[0] not in ("GPU-0f0e-test", "3"):
    print("No devices were found", file=sys.stderr)
    sys.exit(6)
print("3")
'''


@pytest.fixture
def fake_smi_ids(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE_ID.replace("{py}", sys.executable))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    return exe


class _Props:
    def __init__(self, uuid):
        self.uuid = uuid


def test_clock_id_is_the_device_uuid(fake_smi_ids, monkeypatch):
    """torch's cuda:0 is physical GPU 3 here; its UUID names it for nvidia-smi,
    where torch's index 0 would name another GPU."""
    import torch
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3")
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: _Props("0f0e-test"))
    assert bench.smi_device_id(torch.device("cuda", 0)) == "GPU-0f0e-test"


def test_clock_id_from_visible_devices(fake_smi_ids, monkeypatch):
    """Without a UUID the CUDA_VISIBLE_DEVICES entry of the device is used."""
    import torch

    def no_props(d):
        raise RuntimeError("no device")
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,3")
    monkeypatch.setattr(torch.cuda, "get_device_properties", no_props)
    assert bench.smi_device_id(torch.device("cuda", 1)) == "3"


def test_clock_id_falls_back_to_the_index(tmp_path, monkeypatch):
    """No nvidia-smi at all: torch's index, and the sampler reports it unavailable."""
    import torch
    monkeypatch.setenv("PATH", str(tmp_path))
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES", raising=False)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: _Props(""))
    assert bench.smi_device_id(torch.device("cuda", 0)) == "0"


def test_reference_arm_weights_step_rates_by_the_encode(monkeypatch, capsys):
    """The reference line's value is the whole-encode rate: each quadtree
    step's sampled oracle rate weighted by that step's matches in the
    oracle's full encode, not the raw sum over the sample."""
    import argparse
    import json as _json
    rates = [1e7, 4e7, 1e8]                       # matches per second at B = 16, 8, 4

    def fake_sample(img, ss, per_level=(0, 0, 0), seed=0, nthreads=0):
        m, s, d = 0, 0.0, []
        for lvl, k in enumerate(per_level):
            if k:
                mm = k * 1000 * 8
                m += mm
                s += mm / rates[lvl]
                d.append(f"{k} ranges at level {lvl}")
        return m, s, "; ".join(d)

    weights = [2e9, 8e9, 3e10]
    monkeypatch.setattr(bench, "oracle_sample", fake_sample)
    monkeypatch.setattr(bench, "oracle_encode_matches", lambda: [int(w) for w in weights])
    args = argparse.Namespace(steps=2, warmup=3, gpus=1)
    assert bench.run_reference(args) == 0
    line = _json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    want = sum(weights) / sum(w / r for w, r in zip(weights, rates)) / 1e9
    assert line["impl"] == "reference"
    assert abs(line["value"] - want) < 1e-12 * want
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert "oracle's full encode" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_stored_oracle_counts_are_read():
    m = bench.oracle_encode_matches()
    assert m is not None and len(m) == 3 and all(x > 0 for x in m)


def test_fp16_peak_is_the_larger_measured_figure(monkeypatch):
    """The contraction's peak: the larger of the committed FP16 GEMM burst and
    the driver's BF16 burst, so a low FP16 measurement never flatters the
    fraction; with neither, the recipe's fallback, said so."""
    import json
    pk = json.load(open(os.path.join(bench.ROOT, "profiles", "peak_gemm_fp16_bf16.json")))
    fp16 = float(pk["fp16"]["burst_tflops"])
    v, note = bench.fp16_peak({"bf16_tflops": fp16 + 100.0})
    assert v == fp16 + 100.0 and "MEASURED_PEAKS" in note and note.startswith("of measured")
    v, note = bench.fp16_peak({"bf16_tflops": fp16 - 100.0})
    assert v == fp16 and "peak_gemm_fp16_bf16" in note
    real_open = open

    def no_profile(path, *a, **k):
        if str(path).endswith("peak_gemm_fp16_bf16.json"):
            raise FileNotFoundError(path)
        return real_open(path, *a, **k)
    monkeypatch.setattr("builtins.open", no_profile)
    v, note = bench.fp16_peak({})
    assert v == 1900.0 and note.startswith("of fallback")


class _Res:
    def __init__(self, N, ranges):
        self.N, self.ranges = N, ranges


def test_entropy_updates_count():
    """Per run of 32 positions one full window of (2B)^2 pixels, then
    2 min(L, 2B) 2B updates per further position; steps no range reached
    count nothing."""
    # N = 64, L = 2: B = 16 -> per = (64 - 32) / 2 + 1 = 17 (one run per row)
    r = _Res(64, [16, 0, 0])
    assert bench.entropy_updates([r], L=2, B_max=16) == 17 * 32 * 32 + (17 * 17 - 17) * 2 * 2 * 32
    # L = 40 >= 2B = 32 at B = 16: the whole window is replaced per position
    r = _Res(96, [9, 4, 0])
    per16 = (96 - 32) // 40 + 1
    per8 = (96 - 16) // 40 + 1
    want = per16 * 32 * 32 + (per16 * per16 - per16) * 2 * 32 * 32 + \
        per8 * 16 * 16 + (per8 * per8 - per8) * 2 * 16 * 16
    assert bench.entropy_updates([r], L=40, B_max=16) == want


def test_contraction_only_uses_the_capture_while_sources_match(monkeypatch):
    prof = bench.contraction_profile()
    if prof is None:
        pytest.skip("kernel sources changed since the committed capture")
    flops = [1e12, 1e12, 1e12]
    co = bench.contraction_only(flops, 2000.0)
    act = sum(x["duration_ms_under_ncu"] * x["tensor_pipe_active_pct"] / 100.0
              for x in prof["launches"])
    assert co["tflops_while_tensor_pipe_active"] == pytest.approx(3e12 / (act / 1e3) / 1e12)
    assert co["frac"] == pytest.approx(co["tflops_while_tensor_pipe_active"] / 2000.0)
    assert bench.contraction_only(flops[:2], 2000.0) is None
    monkeypatch.setattr(bench, "contraction_profile", lambda: None)
    assert bench.contraction_only(flops, 2000.0) is None and bench.measured_traffic() is None
