"""The JSON line bench.py prints, checked on the reference arm (the CPU
oracle, which runs without a GPU): one line, the contract's keys and types,
the same metric, unit and workload description as the native arm."""
import ctypes
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as wl  # noqa: E402


def test_default_inner_tolerance_is_the_librarys():
    from paper_1602_05650_gb300 import _native, build
    build.build()
    o = _native.fs_options()
    assert _native.load().fs_options_default(ctypes.byref(o)) == 0
    assert bench.DEFAULT_INNER_TOL == o.inner_tol


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("implicit steps/s (" + bench.WORKLOAD)
    assert d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["scaling"] == "weak" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(1e3 / d["value"])
    # the same workload description as the native arm at its defaults
    assert d["config"] == bench.workload_config(wl.cfg_cloud_mixed(0), 1, bench.DEFAULT_INNER_TOL, 1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["cpu"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
