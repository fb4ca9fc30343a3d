"""Host-side parts of bench.py on CPU: the reference arm (the FP64 oracle on
the host cores) prints one JSON line with the keys the bench contract needs,
and a stored ncu traffic figure is used only while the kernel source it was
taken from is unchanged."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("fname", ["traffic.json", "traffic_k_plain.json"])
def test_stored_traffic_only_for_its_kernel_source(fname):
    import bench
    with open(os.path.join(ROOT, "profiles", fname)) as f:
        tj = json.load(f)
    assert bench.stored_traffic(fname, tj["kernel_desc"], tj["source_sha"]) == tj["bytes_per_launch"]
    assert bench.stored_traffic(fname, tj["kernel_desc"], "0" * 16) is None
    assert bench.stored_traffic(fname, tj["kernel_desc"] + " other", tj["source_sha"]) is None
    assert bench.stored_traffic("no_such_file.json", tj["kernel_desc"], tj["source_sha"]) is None


def test_kernel_source_hashes_are_stable():
    import bench
    for fn in (bench.tc_kernel_sha, bench.plain_kernel_sha):
        h = fn()
        assert h == fn() and len(h) == 16 and int(h, 16) >= 0
    assert bench.tc_kernel_sha() != bench.plain_kernel_sha()
