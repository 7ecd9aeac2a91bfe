"""Host logic of bench.py without a GPU: the reference arm's JSON line (the
oracle on the host cores) carries the keys the benchmark contract asks for
and the same config object as the GPU arm, and the DRAM-traffic lookup
takes the ratio recorded for the exact kernel source digest only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_reference_arm_line(bench):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "pairs/s"
    assert d["value"] > 0 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["config"] == bench.bench_config(1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_recorded_traffic_takes_the_exact_digest(bench, tmp_path, monkeypatch):
    dig = bench.kernel_source_digest("k_bfs")
    f = tmp_path / "traffic.txt"
    f.write_text("# comment k_bfs %s 9.0\n" % dig + "k_bfs 0000000000000000 7.0\n" + "k_bfs %s 1.25\n" % dig)
    monkeypatch.setattr(bench, "TRAFFIC", str(f))
    assert bench.recorded_traffic("k_bfs", 4.0e9) == pytest.approx(5.0e9)
    assert bench.recorded_traffic("k_bfs@large", 4.0e9) is None       # a workload variant needs its own line
    assert bench.recorded_traffic("k_pfm_cta", 4.0e9) is None
    f.write_text("k_bfs@large %s 2.0\n" % dig)
    assert bench.recorded_traffic("k_bfs@large", 4.0e9) == pytest.approx(8.0e9)
    f.write_text("k_bfs 0000000000000000 5.0\n")                      # another source's ratio
    assert bench.recorded_traffic("k_bfs", 4.0e9) is None
