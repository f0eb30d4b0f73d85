"""The JSON line of bench.py's reference arm (the FP64 oracle on the host
cores; CPU only).

The line carries the keys a reader of the benchmark output relies on, with
`impl` "reference", a `cpu_baseline` describing the run and an end-to-end
figure that equals the line's own (the oracle moves no data to a device).
Launched as a non-zero rank, the arm does no work and prints nothing.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=timeout)
    assert res.returncode == 0, res.stderr[-2000:]
    return [l for l in res.stdout.splitlines() if l.strip()]


@pytest.mark.parametrize("workload,extra", [("cine", []), ("paper", []), ("cine", ["--storage", "bf16"])],
                         ids=["cine", "paper", "cine-bf16"])
def test_reference_line(workload, extra):
    out = _run(["--impl", "reference", "--workload", workload, "--steps", "1", "--warmup", "3"] + extra)
    assert len(out) == 1
    line = json.loads(out[0])
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["steps"] == 1 and line["warmup"] == 3
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    if extra:  # the reference arm describes the configuration of the arm it is compared with
        assert "BF16" in line["config"]["workload"] and "bfloat16" in line["config"]["storage"]


def test_reference_other_ranks_do_nothing():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"],
               env_extra={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, timeout=60)
    assert out == []
