"""The reference arm of the benchmark (the oracle on the host cores) prints one
JSON line with the contract's keys and the same metric, unit and config as the
native arm's line for the workload; workloads without an oracle arm print an
`unavailable` line and exit 0.  Runs on the CPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_reference_arm_line_small_workload(oracle_mod):
    import bench
    import synth

    d = _run("--workload", "small_u8", "--steps", "1", "--warmup", "3", "--cpu-rows", "64", "--cpu-planes", "1")
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    acq = synth.CONFIGS[bench.WORKLOADS["small_u8"][0]]
    want = bench.single_config("small_u8", acq, acq.side_a, acq.side_a, acq.side_b, acq.side_b,
                               bench.WORKLOADS["small_u8"][1], 1)
    assert d["config"] == want


def test_reference_arm_unavailable_for_workloads_without_an_oracle_arm():
    d = _run("--workload", "denoise", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and "unavailable" in d
