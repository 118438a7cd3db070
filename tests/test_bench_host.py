"""Host-side parts of bench.py (CPU): the DRAM-traffic table's guard and the
reference arm's JSON line.

The traffic table scales a kernel's algorithmic bytes by the DRAM bytes per
algorithmic byte of one ncu capture, and must stop doing so as soon as the
kernel's source (or a shared device header) differs from the captured one.
The reference arm times the CPU oracle and prints the contract's
``"impl": "reference"`` line on rank 0 only.
"""
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_table_entries_are_well_formed():
    assert bench.TRAFFIC_PER_ALGO_BYTE, "no captured kernel"
    for kernel, (path, sha, ratio) in bench.TRAFFIC_PER_ALGO_BYTE.items():
        assert os.path.exists(os.path.join(ROOT, path)), path
        assert re.fullmatch(r"[0-9a-f]{40}", sha), (kernel, sha)
        # DRAM traffic cannot undercut the bytes the kernel must move
        assert 1.0 <= ratio < 50.0, (kernel, ratio)
        got = bench.traffic_for(kernel, 1000.0)
        assert got is None or got == pytest.approx(ratio * 1000.0)
    for header in bench.KERNEL_HEADERS:
        assert os.path.exists(os.path.join(ROOT, header)), header


def test_traffic_applies_only_to_the_captured_source(monkeypatch):
    kernel, (path, sha, ratio) = next(iter(bench.TRAFFIC_PER_ALGO_BYTE.items()))
    current = bench.kernel_source_sha(path)
    monkeypatch.setitem(bench.TRAFFIC_PER_ALGO_BYTE, kernel, (path, current, ratio))
    assert bench.traffic_for(kernel, 10.0) == pytest.approx(10.0 * ratio)
    stale = ("0" if current[0] != "0" else "1") + current[1:]
    monkeypatch.setitem(bench.TRAFFIC_PER_ALGO_BYTE, kernel, (path, stale, ratio))
    assert bench.traffic_for(kernel, 10.0) is None
    monkeypatch.setitem(bench.TRAFFIC_PER_ALGO_BYTE, kernel, (path, None, ratio))
    assert bench.traffic_for(kernel, 10.0) is None
    assert bench.traffic_for("no_such_kernel", 10.0) is None


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                           "tiny", "--steps", "2", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=300)


def test_reference_arm_prints_the_contract_line():
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 3
    assert line["config"]["workload"] == "tiny"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
