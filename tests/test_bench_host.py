"""The host-side contract of bench.py that needs no GPU: the reference arm
(the FP64 oracle on the host cores) and the one-core sample print the JSON
the benchmark's consumers read."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, env=None):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_reference_arm_prints_the_contract_line():
    line = run_bench("--impl", "reference", "--workload", "couette_fp64", "--steps", "2", "--warmup", "3")
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "couette_rigid_sphere_32^3_fp64" and line["config"]["cells"] == 32 ** 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_one_core_sample_runs_the_oracle_on_one_thread():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = run_bench("--cpu-sample", "0.5", "--workload", "couette_fp64", env=env)
    assert out["cores"] == 1 and out["kind"] == "oracle" and out["value"] > 0
    assert out["sample"].startswith("2 steps") or int(out["sample"].split()[0]) >= 2
