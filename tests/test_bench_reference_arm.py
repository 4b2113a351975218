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

    d = _run("--workload", "small_u8", "--steps", "2", "--warmup", "3")
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    # steps and ms_per_step are what was timed: their product fits the timed region
    assert d["steps"] == 2 and d["steps"] * d["ms_per_step"] / 1e3 <= d["wall_s_timed_region"] * 1.001
    assert "sampled" not in d            # the whole step
    acq = synth.CONFIGS[bench.WORKLOADS["small_u8"][0]]
    want = bench.single_config("small_u8", acq, acq.side_a, acq.side_a, acq.side_b, acq.side_b,
                               bench.WORKLOADS["small_u8"][1], 1)
    assert d["config"] == want


def test_reference_arm_unavailable_for_workloads_without_an_oracle_arm():
    d = _run("--workload", "denoise", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and "unavailable" in d


def test_oracle_step_sample_is_the_proportional_part_of_the_step(oracle_mod):
    """The sampled reference step (the default workload's) computes the Gamma rows
    of the first k spatial image rows, bit-identical to those rows of the whole
    oracle step, the same fraction k / H_a of the planes, and counts the
    sample's own operations."""
    import numpy as np

    import bench
    import synth

    acq = synth.Acquisition(12, 6, 300, 2.0, "poisson8", seed=5)
    A, B = synth.generate(acq, "cpu")
    fr, lay = synth.pack_side_by_side(A, B, 8)
    host = fr.numpy()
    alpha, beta = synth.uniform_planes(24)
    g_ref = bench.synth_gamma(144, 36)
    t, ops, desc, r, ref = bench.oracle_step(acq, (alpha, beta), host, lay, 2, g_ref)
    full = oracle_mod.correlate(host, lay["a"], host, lay["b"], acq.n_frames)
    assert ops == 2.0 * 24 * 36 * acq.n_frames and t > 0
    assert np.array_equal(r["s_ab"], full["s_ab"][:24])
    assert np.array_equal(r["gamma"].view(np.int64), full["gamma"][:24].view(np.int64))
    assert ref.shape == (4, 12, 12)            # 24 planes x 2 / 12 rows
    assert np.array_equal(ref, oracle_mod.refocus(g_ref, 12, 12, 6, 6, alpha[:4], beta[:4]))
