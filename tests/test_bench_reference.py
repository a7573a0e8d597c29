"""bench.py's reference arm (the oracle timed on the host cores) and its JSON line, on the CPU.

It must describe the same workload, metric, unit and direction as the GPU arm, report the oracle's sample
and thread count, and leave every rank but 0 without work under a multi-rank launch."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line_matches_the_gpu_arm_contract():
    import bench
    p = _run({}, "--workload", "shear32_v24_nh1_fp64", "--steps", "1", "--warmup", "3")
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    cases = bench.workloads()["shear32_v24_nh1_fp64"]()
    upd = sum(c.updates_per_iteration() for c in cases)
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["config"] == bench.describe("shear32_v24_nh1_fp64", cases, upd, 1)
    assert line["steps"] == 1 and line["warmup"] >= 3 and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["host"]["nproc"] >= 1 and cb["host"]["machine"]
    assert cb["cores"] == bench.usable_cores() == line["sample_config"]["processes"]
    sc = line["sample_config"]                     # what each step actually ran
    assert sc["cells"] == [8, 8] and sc["velocities"] == [24, 24] and sc["n_levels"] == 3
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    p = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "3")
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
