"""GPU parity of the Eq. (1) finalisation on arbitrary integer sums.

Gamma = (double)(N*S_ab - S_a*S_b) / ((double)N * (double)N) with IEEE
round-to-nearest conversion and division; numpy performs exactly those two
operations, so the kernel's result must match bit for bit, including numerators
next to powers of two (where the spacing of doubles changes) and the frame
counts that take the kernel's general division path."""

import numpy as np
import pytest
import torch

import paper_2407_20692_gb300 as cpi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready):
    yield


def _expected(num, n):
    d = np.float64(n) * np.float64(n)
    return num.astype(np.float64) / d


@pytest.mark.parametrize("n", [1, 2, 3, 7, 1000, 20000, 50000, 1_048_577, 67_108_863, 100_000_001])
def test_finalize_random_and_boundary_numerators(n):
    rng = np.random.default_rng(n)
    ma, mb = 64, 96
    # rows with s_a = 1: num = n * s_ab + r, r a random residue (s_b = -r)
    lim = min((1 << 62) // max(n, 1), 1 << 40)
    s_ab = rng.integers(-lim, lim, size=(ma, mb), dtype=np.int64)
    r = rng.integers(0, max(n, 1), size=mb, dtype=np.int64)
    s_a = np.ones(ma, dtype=np.int64)
    # rows 0..k with s_a = 0: num = n * s_ab, quotient s_ab / n placed next to 2^k
    # (where the spacing of doubles changes): s_ab = n 2^k + delta, |delta| <= 3
    for i, k in enumerate(range(-20, 30, 5)):
        base = (n << k) if k >= 0 else (n >> (-k))
        if base * n >= 1 << 61 or base < 4:
            continue
        s_a[i] = 0
        for j in range(mb):
            s_ab[i, j] = base + (j % 7) - 3
    s_b = -r
    num = n * s_ab - s_a[:, None] * s_b[None, :]
    dev = "cuda"
    g = torch.empty((ma, mb), dtype=torch.float64, device=dev)
    g32 = torch.empty((mb, ma), dtype=torch.float32, device=dev)
    cpi.cpi_correlate_finalize(torch.from_numpy(s_ab).to(dev), torch.from_numpy(s_a).to(dev),
                               torch.from_numpy(s_b).to(dev), ma, mb, n, g, g32)
    torch.cuda.synchronize()
    want = _expected(num, n)
    got = g.cpu().numpy()
    bad = np.argwhere(got.view(np.int64) != want.view(np.int64))
    assert len(bad) == 0, (len(bad), bad[:3], got[tuple(bad[0])], want[tuple(bad[0])])
    assert np.array_equal(g32.cpu().numpy(), want.astype(np.float32).T)


def test_finalize_zero_and_sign():
    n = 10
    s_ab = torch.tensor([[0, 1, -1], [5, -5, 7]], dtype=torch.int64, device="cuda")
    s_a = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    s_b = torch.tensor([0, 3, 0], dtype=torch.int64, device="cuda")
    g = torch.empty((2, 3), dtype=torch.float64, device="cuda")
    cpi.cpi_correlate_finalize(s_ab, s_a, s_b, 2, 3, n, g, None)
    torch.cuda.synchronize()
    num = 10 * s_ab.cpu().numpy() - np.outer(s_a.cpu().numpy(), s_b.cpu().numpy())
    assert np.array_equal(g.cpu().numpy(), _expected(num, n))
    assert not np.signbit(g.cpu().numpy()[0, 0])
