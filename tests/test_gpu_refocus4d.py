"""GPU parity of the 4-D multilinear refocusing against its FP64 oracle.

Tolerance, per unit of interpolation weight as for the 2-D refocusing:
|R_gpu - R_fp64| <= 1e-6 max|Gamma| W_p(x), W_p(x) the total in-grid weight
(the refocusing of an all-ones Gamma).  The kernels' error: Gamma rounded to FP32
(u/2), four weight fractions rounded to 24 bits (u each), the 4-tap column
sample in FP32 (about 4u of the summed terms), Kahan sums over the angular
columns (2u), the column sums kept as float pairs, the row stage in double-float
FP32 (exact up to the final rounding, u/2): about 11u, 6.6e-7."""

import numpy as np
import pytest
import torch

import oracle
import paper_2407_20692_gb300 as cpi
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready, oracle_mod):
    yield


def _gpu4d(g32, ha, wa, hb, wb, co):
    planes = cpi.plane4_array(*co)
    out = torch.empty((len(co[0]), ha, wa), dtype=torch.float32, device="cuda")
    ws = torch.empty(cpi.cpi_refocus4d_workspace_size(ha, wa, hb, wb, len(co[0])), dtype=torch.uint8, device="cuda")
    cpi.cpi_refocus4d(g32, ha, wa, hb, wb, planes, out, ws)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    return out.cpu().double().numpy()


_CO = (np.array([0.6, 1.0, 1.3, 0.9, 1.0]), np.array([0.4, 0.0, -0.3, 0.25, 0.0]),
       np.array([0.3, 0.0, -0.45, 0.7, 0.0]), np.array([0.8, 1.0, 1.2, 0.5, 1.0]))


@pytest.mark.parametrize("ha,wa,hb,wb", [
    (7, 9, 4, 5),          # ragged, box in shared memory
    (16, 12, 6, 8),
    (2, 260, 2, 200),      # box too large for shared memory: global-memory path
    (33, 17, 3, 2),
    (12, 100, 5, 6),       # two planes per column pass, the last pass ragged
    (9, 300, 3, 4),        # wider than a CTA's threads: columns loop
    (50, 12, 60, 10),      # four row pairs per CTA, the last group of two
    (41, 9, 40, 7),        # two row pairs per CTA, the last group of one
])
def test_refocus4d_random_gamma_matches_oracle(ha, wa, hb, wb):
    rng = np.random.default_rng(ha * 100 + wa)
    gamma = rng.standard_normal((ha * wa, hb * wb))
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    got = _gpu4d(g32, ha, wa, hb, wb, _CO)
    want = oracle.refocus4d(gamma.astype(np.float32).astype(np.float64), ha, wa, hb, wb, *_CO)
    W = oracle.refocus4d(np.ones_like(gamma), ha, wa, hb, wb, *_CO)
    tol = 1e-6 * np.abs(gamma).max() * W
    err = np.abs(got - want)
    assert (err <= tol).all(), (err / np.maximum(tol, 1e-300)).max()


def test_refocus4d_with_gamma0_delta1_is_the_2d_refocusing_on_the_bench_shape():
    """64x64 vs 32x32: the 4-D kernels with gamma = 0, delta = 1 against the 2-D
    refocusing kernels (both within 1e-6 max|Gamma| W of the FP64 result)."""
    ha = wa = 64
    hb = wb = 32
    rng = np.random.default_rng(5)
    gamma = rng.standard_normal((ha * wa, hb * wb)).astype(np.float32)
    g32 = torch.tensor(gamma.T, device="cuda").contiguous()
    alpha, beta = synth.uniform_planes(8)
    got4 = _gpu4d(g32, ha, wa, hb, wb, (alpha, beta, np.zeros(8), np.ones(8)))
    out2 = torch.empty((8, ha, wa), dtype=torch.float32, device="cuda")
    ws = torch.empty(cpi.cpi_refocus_workspace_size(ha, wa, hb, wb, 8), dtype=torch.uint8, device="cuda")
    cpi.cpi_refocus(g32, ha, wa, hb, wb, cpi.plane_array(alpha, beta), out2, ws)
    torch.cuda.synchronize()
    W = oracle.refocus(np.ones((ha * wa, hb * wb)), ha, wa, hb, wb, alpha, beta)
    tol = 2e-6 * np.abs(gamma).max() * W
    assert (np.abs(got4 - out2.cpu().double().numpy()) <= tol).all()


def test_refocus4d_more_planes_than_one_chunk():
    ha, wa, hb, wb = 10, 8, 3, 4
    rng = np.random.default_rng(6)
    gamma = rng.standard_normal((ha * wa, hb * wb))
    g32 = torch.tensor(gamma.T.astype(np.float32), device="cuda").contiguous()
    P = 150
    a = np.linspace(0.5, 1.5, P)
    co = (a, 1.0 - a, 0.5 * (a - 1.0), 1.0 - 0.5 * (a - 1.0))
    got = _gpu4d(g32, ha, wa, hb, wb, co)
    want = oracle.refocus4d(gamma.astype(np.float32).astype(np.float64), ha, wa, hb, wb, *co)
    W = oracle.refocus4d(np.ones_like(gamma), ha, wa, hb, wb, *co)
    assert (np.abs(got - want) <= 1e-6 * np.abs(gamma).max() * W).all()


def test_refocus4d_argument_errors():
    g = torch.zeros(64, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_refocus4d(g, 4, 4, 2, 2, cpi.plane4_array([1.0], [0.0], [2e6], [1.0]), g, ws)
    assert e.value.code == 1
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_refocus4d(g, 0, 4, 2, 2, cpi.plane4_array([1.0], [0.0], [0.0], [1.0]), g, ws)
    assert e.value.code == 1
