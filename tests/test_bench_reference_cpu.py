"""bench.py --impl reference: the FP64 oracle timed on the host cores prints
one JSON line with the benchmark's metric, unit and the keys the benchmark
contract asks of the reference arm. The test runs it on the starfish workload
(--config 2, about 15 s on CPU); the default line is the 200-ellipse workload."""
import json
import os
import subprocess
import sys

from tests.conftest import ROOT


def test_reference_arm_json_line():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--config", "2"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("QBX-FMM layer-potential targets/sec")
    assert d["unit"] == "targets/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("starfish-k10")


def test_default_workload_is_the_ellipses():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.CONFIG_NUM == 5
    assert "200 ellipses" in bench.WORKLOADS[5]
