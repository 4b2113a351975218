"""GPU parity of refocusing against the FP64 oracle.

Tolerance: every refocused value is a sum of bilinear samples of Gamma, so the
error is bounded per unit of interpolation weight: |R_gpu - R_fp64| <=
1e-6 * max|Gamma| * W_p(x), where W_p(x) is the total in-grid interpolation
weight at that output (the refocus of an all-ones Gamma).  The FP32 path has
Gamma rounded to FP32 (2^-24 relative), FP32 weights and products (a few
2^-24), and compensated summation (2 * 2^-24 plus second-order terms), about
5e-7 per unit weight in the worst case."""

import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import gpu_correlate, make_frames, refocus_errors, refocus_gpu, refocus_tolerance

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready, oracle_mod):
    yield


def test_refocus_hand_worked():
    g = json.load(open(os.path.join(GOLD, "refocus_hand.json")))
    gamma = np.array(g["gamma"], dtype=np.float64)
    g32 = torch.tensor(gamma.T.copy(), dtype=torch.float32, device="cuda")
    al = [p[0] for p in g["planes"]]
    be = [p[1] for p in g["planes"]]
    out = refocus_gpu(g32, g["ha"], g["wa"], g["hb"], g["wb"], al, be)
    assert np.array_equal(out, np.array(g["out"]))


@pytest.mark.parametrize("ha,wa,hb,wb", [
    (9, 12, 4, 6),        # 2-D staging, 8 planes per unit
    (64, 64, 32, 32),     # compile-time 64 x 64 shape
    (33, 70, 7, 5),       # width 2 mod 4: 2-D staging from a row-padded copy
    (17, 33, 5, 3),       # width 1 mod 4
    (46, 95, 4, 4),       # width 3 mod 4, 2 planes per unit
    (31, 247, 2, 3),      # widest row-padded 2-D box (248 + 8 columns)
    (7, 249, 2, 2),       # padded row too wide for a 2-D box: 1-D staging
    (5, 300, 3, 2),       # 1-D staging, width above 256
    (96, 96, 8, 8),       # one plane per unit, 32 rows per thread
    (72, 72, 6, 6),       # one plane per unit, 16 rows per thread
    (100, 90, 3, 3),      # one plane per unit, row-padded copy
    (128, 128, 4, 4),     # one plane per unit, two staged slices
    (200, 120, 2, 2),     # 50 rows per thread: direct kernel
])
def test_refocus_random_gamma(ha, wa, hb, wb):
    rng = np.random.default_rng(ha * 1000 + wa)
    gamma = rng.standard_normal((ha * wa, hb * wb))
    alpha = np.array([0.5, 0.77, 1.0, 1.0, 1.31, 1.5, 2.5])
    beta = np.array([0.5, 0.23, 0.0, 0.4, -0.31, -0.5, 1.7])
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    out = refocus_gpu(g32, ha, wa, hb, wb, alpha, beta)
    ref = oracle.refocus(gamma.astype(np.float32).astype(np.float64), ha, wa, hb, wb, alpha, beta)
    literal, per_w, tol = refocus_errors(out, ref, gamma, ha, wa, hb, wb, alpha, beta)
    print(f"refocus {ha}x{wa} vs {hb}x{wb}: max err / max|Gamma| = {literal:.3e}, per unit weight {per_w:.3f}")
    assert (np.abs(out - ref) <= tol).all(), per_w
    assert literal <= 1e-6


def test_refocus_large_u8_shape_sampled_planes():
    """The 128x128 vs 64x64 shape of the 8-bit workload: M_b = 4096 angular
    pixels per output (the longest FP32 sum of the configurations), all 128
    uniformly spaced planes in one call as the benchmark runs them, compared with
    the FP64 oracle on sampled planes (both ends, the middle and two seeded ones)
    of a seeded random Gamma."""
    ha = wa = 128
    hb = wb = 64
    rng = np.random.default_rng(4096)
    gamma = rng.standard_normal((ha * wa, hb * wb)).astype(np.float32).astype(np.float64)
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    alpha, beta = synth.uniform_planes(128)
    out = refocus_gpu(g32, ha, wa, hb, wb, alpha, beta)
    del g32
    idx = sorted({0, 63, 64, 127, *rng.choice(128, 2, replace=False).tolist()})
    ref = oracle.refocus(gamma, ha, wa, hb, wb, alpha[idx], beta[idx])
    literal, per_w, tol = refocus_errors(out[idx], ref, gamma, ha, wa, hb, wb, alpha[idx], beta[idx])
    print(f"refocus 128x128 vs 64x64, planes {idx}: max err / max|Gamma| = {literal:.3e}, per unit weight {per_w:.3f}")
    assert (np.abs(out[idx] - ref) <= tol).all(), per_w
    assert literal <= 1e-6


def test_refocus_spad_1bit_workload():
    """Gamma of the 64x64 vs 32x32 binary workload (20000 frames), 32 uniformly
    spaced planes, against the oracle refocusing the oracle's FP64 Gamma."""
    acq = synth.CONFIGS["spad_1bit"]
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], acq.n_frames)
    want = oracle.correlate(fr.cpu().numpy(), lay["a"], fr.cpu().numpy(), lay["b"], acq.n_frames)
    alpha, beta = synth.uniform_planes(32)
    out = refocus_gpu(got["gamma_f32"], 64, 64, 32, 32, alpha, beta)
    ref = oracle.refocus(want["gamma"], 64, 64, 32, 32, alpha, beta)
    literal, per_w, tol = refocus_errors(out, ref, want["gamma"], 64, 64, 32, 32, alpha, beta)
    print(f"refocus of the 64x64 vs 32x32 binary workload's Gamma: max err / max|Gamma| = {literal:.3e}, "
          f"per unit weight {per_w:.3f}")
    assert (np.abs(out - ref) <= tol).all(), per_w
    assert literal <= 1e-6


def test_refocus_focused_plane_row_sums():
    acq = synth.Acquisition(16, 16, 2000, 2.0, "poisson8", seed=8)
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], acq.n_frames)
    out = refocus_gpu(got["gamma_f32"], 16, 16, 16, 16, [1.0], [0.0])
    rows = got["gamma"].numpy().sum(1).reshape(16, 16)
    tol = 1e-6 * np.abs(got["gamma"].numpy()).max() * 256
    assert np.abs(out[0] - rows).max() <= tol


def test_refocus_many_planes_two_launches():
    """More planes than one launch carries (128): results must not depend on it."""
    rng = np.random.default_rng(3)
    ha, wa, hb, wb = 12, 10, 3, 4
    gamma = rng.standard_normal((ha * wa, hb * wb))
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    alpha, beta = synth.uniform_planes(200)
    out = refocus_gpu(g32, ha, wa, hb, wb, alpha, beta)
    ref = oracle.refocus(gamma.astype(np.float32).astype(np.float64), ha, wa, hb, wb, alpha, beta)
    tol = refocus_tolerance(gamma, ha, wa, hb, wb, alpha, beta)
    assert (np.abs(out - ref) <= tol).all()
