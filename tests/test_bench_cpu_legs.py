"""The benchmark's CPU legs run here without a GPU: the reference arm (the
oracle timed on the host) prints one JSON line with the contract's keys, and
the CPU baseline reports Algorithm 1 on all cores, one core and the naive
definition per window."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-sample", "65536"], capture_output=True, text=True, cwd=ROOT,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Gelem/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "Gelem/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("long 1D stream")


def test_cpu_baseline_fields():
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.cpu_baseline(1 << 16)
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["single_core_value"] > 0
    naive = cb["naive_single_core_by_window"]
    assert sorted(naive, key=int) == [str(w) for w in bench.WINDOWS if w <= 1001]
    assert all(v["value"] > 0 and v["sample"] > 0 for v in naive.values())
    # the naive definition costs 2w-2 comparisons per output: slower as w grows
    assert naive["3"]["value"] > naive["1001"]["value"]
