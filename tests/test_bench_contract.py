"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the JSON-line
contract: one line with impl = reference, the same metric as the GPU arm, a positive time
(each timed step one complete oracle solve), the CPU-baseline description and an end-to-end
entry with no host-device traffic.  Ranks
other than 0 print nothing.  Runs on the CPU at 32^3."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "1", "--n", "32"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = run_bench()
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "ms" and d["value"] > 0 and d["higher_is_better"] is False
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n"] == 32 and d["config"]["oracle_iters"] > 0
    # each timed step is one complete solve: the timed region holds exactly steps x value
    assert abs(d["config"]["timed_region_s"] * 1e3 - d["steps"] * d["value"]) <= 0.05 * d["steps"] * d["value"] + 5


def test_reference_arm_is_silent_off_rank_zero():
    r = run_bench({"RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
