"""The benchmark's reference arm (the FP64 oracle on the host cores, a thread
per core over independent runs) prints one JSON line with the fields of the
benchmark contract; a small manifest keeps it to seconds on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--runs", "4", "--scale", "0.02", "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "particle-steps/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps_timed"] == 3 and line["warmup_done"] == 1
    cb = line["cpu_baseline"]
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # a thread per host core, at most one per run of the 4-run sample
    assert cb["kind"] == "oracle" and cb["cores"] == min(threads, 4)
    assert cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0
