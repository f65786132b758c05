"""The benchmark's output contract, on CPU: the reference arm (the FP64 oracle
on the host cores) prints one JSON line with every key the line must carry,
and the measured DRAM-traffic and FP64-instruction counters are reported only
for the kernel source they were taken on."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] in ("weak", "strong")
    assert d["vs_baseline"] is None and d["data"] == "synthetic" and d["dtype"] == "f64"
    assert d["config"]["workload"] == bench.WORKLOAD
    # the line reports what was timed: the sample's columns, K steps of it
    c = d["config"]
    assert c["ncols"] % 32 == 0 and 0 < c["ncols"] <= c["sample_of_ncols"]
    assert d["ms_per_step"] * d["steps"] == pytest.approx(c["timed_s"] * 1e3, rel=1e-9)
    assert d["value"] == pytest.approx(c["ncols"] * c["nlev"] / (d["ms_per_step"] * 1e-3), rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_measured_counters_follow_the_kernel_source(monkeypatch):
    with open(os.path.join(ROOT, bench.MEASURED_TRAFFIC["source"]), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    npts = 39_321_600
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "sha256", sha)
    monkeypatch.setitem(bench.MEASURED_FP64_OPS, "sha256", sha)
    # the captured launch's own bytes at its size, per point elsewhere
    assert bench._measured_traffic(npts) == bench.MEASURED_TRAFFIC["bytes_per_launch"]
    assert bench._measured_traffic(npts // 4) == pytest.approx(bench.MEASURED_TRAFFIC["bytes_per_point"] * npts // 4)
    # the DFMA rate is probed on the GPU at run time; here a fixed stand-in
    from paper_2010_14823_gb300 import peaks
    monkeypatch.setattr(peaks, "peak_rate", lambda kind, iters: 0.5e12)
    r = bench._fp64_roofline(npts, 139.0)
    assert r["achieved"] == pytest.approx(bench.MEASURED_FP64_OPS["inst_per_point"] * npts / 0.139)
    assert r["frac"] == pytest.approx(r["achieved"] / 0.5e12)
    # a different source: neither counter is reported
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "sha256", "0" * 64)
    monkeypatch.setitem(bench.MEASURED_FP64_OPS, "sha256", "0" * 64)
    assert bench._measured_traffic(npts) is None
    assert bench._fp64_roofline(npts, 139.0) is None
