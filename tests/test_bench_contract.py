"""bench.py's command-line contract, on the CPU: the reference arm (the oracle timed
on host cores) prints one JSON line with the fields the contract names, only rank 0
prints under a multi-rank launch, and the default step counts per mode."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return out.stdout


@pytest.mark.parametrize("workload,needle", [("walks", "random walks"), ("mixed", "mixed shapes")])
def test_reference_arm_prints_one_contract_line(workload, needle):
    out = _run(["--impl", "reference", "--workload", workload, "--n", "200000", "--cpu-sample", "20000",
                "--cpu-queries", "2", "--queries", "4", "--steps", "1", "--warmup", "1"])
    lines = [l for l in out.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "queries/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "20000 of the 200000" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert needle in d["config"]["workload"] and d["data"] == "synthetic" and d["vs_baseline"] is None


def test_reference_arm_is_silent_off_rank_zero():
    out = _run(["--impl", "reference", "--n", "200000", "--cpu-sample", "20000", "--cpu-queries", "1",
                "--steps", "1", "--warmup", "1"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert out.strip() == ""


def test_default_steps_per_mode(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for argv, steps in ((["bench.py"], 100), (["bench.py", "--dtw"], 10), (["bench.py", "--serving"], 10),
                        (["bench.py", "--impl", "reference"], 10), (["bench.py", "--steps", "7"], 7)):
        monkeypatch.setattr(sys, "argv", argv)
        args = bench.parse()
        assert args.steps == steps and args.warmup == 3 and args.gpus == 1, argv
