"""The benchmark's reference arm (`bench.py --impl reference`: the FP64 oracle timed on the
host cores) runs without a GPU and prints one JSON line with every key of the benchmark
contract; its metric and workload are the ones the GPU arm reports."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "env-steps/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "humanoid8192"
    # the GPU arm's config for the same arguments: both arms step the same workload state
    assert d["config"] == {"workload": "humanoid8192", "groups": [["humanoid", 8192]], "worlds_per_gpu": 8192,
                           "decimation": 4, "preroll_env_steps": 100, "parallelism": "replicas x1"}
    assert "pre-rolled 100 env steps" in d["cpu_baseline"]["sample"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["gpu_launches"] == 0
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC
