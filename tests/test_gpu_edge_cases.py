"""Degenerate and extreme inputs through the C ABI, against the oracle.

Eq. (1) with a single frame is identically zero (every pixel equals its own
mean); all-zero frames give zero sums and zero Gamma; 1 x 1 detectors reduce the
contraction to one dot product.  Refocusing with one angular pixel is a single
interpolated image; alpha = 0 samples every output at the same point; a plane
whose samples all fall outside the grid gives exactly 0; the widest image the
kernels take (512 columns) runs the direct kernel.  The 4-D refocusing with
gamma = delta = 0 samples one angular point for every output."""

import numpy as np
import pytest
import torch

import oracle
import paper_2407_20692_gb300 as cpi
import synth
from gpu_util import assert_exact, gpu_correlate, make_frames, oracle_correlate, refocus_gpu, refocus_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready, oracle_mod):
    yield


@pytest.mark.parametrize("counts", ["bernoulli", "poisson8"])
def test_single_frame_gives_zero_gamma(counts):
    acq = synth.Acquisition(12, 8, 1, 2.0 if counts == "poisson8" else 0.5, counts, seed=31)
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], 1)
    want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], 1)
    assert_exact(got, want)
    assert not got["gamma"].numpy().any()


@pytest.mark.parametrize("counts", ["bernoulli", "poisson8"])
def test_all_zero_frames(counts):
    acq = synth.Acquisition(16, 8, 700, 1.0, counts, seed=32)
    fr, lay = make_frames(acq)
    fr.zero_()
    got = gpu_correlate(fr, lay["a"], lay["b"], 700)
    for k in ("s_ab", "s_a", "s_b", "gamma"):
        assert not got[k].numpy().any(), k


@pytest.mark.parametrize("counts", ["bernoulli", "poisson8"])
def test_one_by_one_detectors(counts):
    acq = synth.Acquisition(1, 1, 3000, 2.0 if counts == "poisson8" else 0.5, counts, seed=33)
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], 3000)
    want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], 3000)
    assert_exact(got, want)


def _refocus_vs_oracle(gamma, ha, wa, hb, wb, alpha, beta):
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    out = refocus_gpu(g32, ha, wa, hb, wb, alpha, beta)
    ref = oracle.refocus(gamma.astype(np.float32).astype(np.float64), ha, wa, hb, wb, alpha, beta)
    tol = refocus_tolerance(gamma, ha, wa, hb, wb, alpha, beta)
    err = np.abs(out - ref)
    assert (err <= tol).all(), (err / np.maximum(tol, 1e-300)).max()
    return out


def test_refocus_single_angular_pixel():
    rng = np.random.default_rng(34)
    gamma = rng.standard_normal((20 * 24, 1))
    _refocus_vs_oracle(gamma, 20, 24, 1, 1, np.array([0.5, 1.0, 1.3]), np.array([0.5, 0.0, -0.3]))


def test_refocus_alpha_zero_samples_one_point_per_angular_pixel():
    rng = np.random.default_rng(35)
    ha, wa, hb, wb = 9, 12, 4, 5
    gamma = rng.standard_normal((ha * wa, hb * wb))
    out = _refocus_vs_oracle(gamma, ha, wa, hb, wb, np.array([0.0, 0.0]), np.array([0.0, 0.7]))
    # alpha = 0: the output does not depend on the pixel
    for p in range(2):
        assert np.allclose(out[p], out[p][0, 0], rtol=0, atol=1e-6 * np.abs(gamma).max() * hb * wb)


def test_refocus_plane_outside_the_grid_is_exactly_zero():
    rng = np.random.default_rng(36)
    ha, wa, hb, wb = 8, 16, 3, 4
    gamma = rng.standard_normal((ha * wa, hb * wb))
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    out = refocus_gpu(g32, ha, wa, hb, wb, np.array([1.0, 1.0]), np.array([1.0e5, -1.0e5]))
    assert not out.any()


def test_refocus_widest_image():
    rng = np.random.default_rng(37)
    ha, wa, hb, wb = 3, 512, 2, 2
    gamma = rng.standard_normal((ha * wa, hb * wb))
    _refocus_vs_oracle(gamma, ha, wa, hb, wb, np.array([0.8, 1.0, 1.2]), np.array([0.2, 0.0, -0.2]))


def test_refocus4d_single_angular_point():
    rng = np.random.default_rng(38)
    ha, wa, hb, wb = 6, 10, 4, 5
    gamma = rng.standard_normal((ha * wa, hb * wb))
    co = (np.array([1.0, 0.7]), np.array([0.0, 0.3]), np.array([0.0, 0.0]), np.array([0.0, 0.0]))
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    out = torch.empty((2, ha, wa), dtype=torch.float32, device="cuda")
    ws = torch.empty(cpi.cpi_refocus4d_workspace_size(ha, wa, hb, wb, 2), dtype=torch.uint8, device="cuda")
    cpi.cpi_refocus4d(g32, ha, wa, hb, wb, cpi.plane4_array(*co), out, ws)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    want = oracle.refocus4d(gamma.astype(np.float32).astype(np.float64), ha, wa, hb, wb, *co)
    W = oracle.refocus4d(np.ones_like(gamma), ha, wa, hb, wb, *co)
    assert (np.abs(out.cpu().double().numpy() - want) <= 1e-6 * np.abs(gamma).max() * W).all()
