"""bench.py's host-side legs run without a GPU: the reference arm (the
oracle on the host cores) prints its JSON line, and the cpu_baseline leg's
oracle step timer works on a small grid."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "8",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "steps/s"
    assert line["config"]["workload"] == "smooth-mode 8^3"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_step_timer():
    sys.path.insert(0, ROOT)
    import bench
    t, cycles = bench.oracle_step_time(8)
    assert t > 0 and cycles >= 1
