"""bench.py's reference arm (the oracle on the whole matrix of the workload,
one step) on CPU, here on a small scale of the workload: the JSON line of the
contract, for the default method and for the Section 5 preconditioners."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("extra,precond", [([], None), (["--dd", "4", "--overlap", "1"], "ras"),
                                           (["--dd", "4", "--overlap", "0"], "bj"),
                                           (["--dd", "4", "--overlap", "1", "--additive"], "asm"),
                                           (["--dd", "4", "--schur", "3"], "schur")])
def test_reference_arm_line(extra, precond):
    d = _run("--workload", "geo60k_l6", "--scale", "0.007", "--steps", "3", "--warmup", "2", *extra)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "geo60k_l6"
    # one step of the oracle, reported as run (the requested counts are noted)
    assert d["steps"] == 1 and d["warmup"] == 0 and d["cpu_baseline"]["requested_steps"] == 3
    assert d["config"].get("precond") == precond
    if precond:
        assert d["config"]["nparts"] == 4
    if precond == "schur":
        assert d["config"]["inner_steps"] == 3 and "overlap" not in d["config"]
