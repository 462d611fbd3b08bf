"""CPU checks of bench.py's command line and of the reference arm's JSON line
(the reference arm times the oracle on the host's cores, so it runs without a
GPU): one line, the metric and config keys of the own arm, a cpu_baseline with
the cores used, and an e2e entry with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_parse_defaults_and_workloads():
    bench = _bench_module()
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
        assert (a.gpus, a.workload, a.impl, a.precision, a.tile) == (1, "full", "ours", "f64", 16)
        assert a.warmup >= 3
        for wl in ("spatiotemporal", "large", "sweep", "serve", "servebatch"):
            sys.argv = ["bench.py", "--workload", wl]
            assert bench.parse().workload == wl
        sys.argv = ["bench.py", "--workload", "large", "--marginal-variances", "--sweep="]
        a = bench.parse()
        assert a.marginal_variances and a.sweep == ""
    finally:
        sys.argv = old


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-workers", "2"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "TFLOP/s" and d["higher_is_better"] is True
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (1, 0, 1)
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
