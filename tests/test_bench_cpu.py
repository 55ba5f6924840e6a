"""bench.py's reference arm (the FP64 oracle on the host cores) honours the
JSON-line contract (CPU only, small workload)."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_json_line():
    d = run("--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "1")
    for k in ("impl", "metric", "value", "unit", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_reference_arm_unavailable_for_device_only_workloads():
    for wl in ("grad", "protocol", "fairness", "sweep"):
        d = run("--impl", "reference", "--workload", wl)
        assert d["impl"] == "reference" and "unavailable" in d, wl


def test_reference_arm_of_the_grid_workload():
    d = run("--impl", "reference", "--workload", "grid", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "item-rounds/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_workload_table():
    # every workload names its kind's required fields and a description of
    # what it runs (the JSON line's config.workload)
    sys.path.insert(0, ROOT)
    import bench
    need = {None: ("n", "m", "p", "shots", "seed"),
            "grad": ("n", "m", "p", "batch", "lr"),
            "sweep": ("count", "grid", "p", "rounds"),
            "protocol": ("count", "n_values", "d_lo", "d_hi", "S", "p_max"),
            "fairness": ("n", "runs", "shots_per_run", "alpha"),
            "study": ("train", "train_n", "test", "test_n", "p"),
            "grid": ("n", "m", "p", "seed")}
    for name, wl in bench.WORKLOADS.items():
        assert isinstance(wl.get("desc"), str) and wl["desc"], name
        for key in need[wl.get("kind")]:
            assert key in wl, (name, key)
    assert bench.WORKLOADS["study"]["train"] == 20000 and bench.WORKLOADS["study"]["test"] == 2000
    assert bench.WORKLOADS["protocol_scaling"]["n_values"] == list(range(10, 25))


def test_reference_arm_unavailable_for_the_study():
    d = run("--impl", "reference", "--workload", "study")
    assert d["impl"] == "reference" and "unavailable" in d
