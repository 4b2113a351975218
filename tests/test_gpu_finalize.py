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


def _expected_bigint(s_ab, s_a, s_b, n):
    """RN(RN(num) / RN(n * n)) with num = n S_ab - S_a S_b formed in Python's
    unbounded integers (int -> float conversion and float division are both
    correctly rounded in Python)."""
    d = float(n) * float(n)
    out = np.empty(s_ab.shape, dtype=np.float64)
    for i in range(s_ab.shape[0]):
        for j in range(s_ab.shape[1]):
            num = n * int(s_ab[i, j]) - int(s_a[i]) * int(s_b[j])
            out[i, j] = float(num) / d
    return out


@pytest.mark.parametrize("n", [12_000_000, 100_000_003, (1 << 31) - 1])
def test_finalize_sums_beyond_int64_products(n):
    """Sums added over many accumulating calls: S_a * S_b leaves int64 (counts of
    255 over more than ~1.2e7 frames).  Rows 0..7 keep the numerator inside int64
    by cancellation (S_ab = S_a S_b / n plus a small residue), the other rows
    have numerators beyond int64; both must match the big-integer formula bit
    for bit."""
    rng = np.random.default_rng(n % 1000)
    ma, mb = 24, 40
    s_a = rng.integers(200 * n // 2, 255 * n, size=ma, dtype=np.int64)
    s_b = rng.integers(100 * n // 2, 255 * n, size=mb, dtype=np.int64)
    s_a[0] = 255 * n                        # the largest sums: S_a S_b = 65025 n^2 >= 2^63 for n >= 1.2e7
    s_b[0] = 255 * n
    s_ab = np.empty((ma, mb), dtype=np.int64)
    for i in range(ma):
        for j in range(mb):
            prod = int(s_a[i]) * int(s_b[j])
            if i < 8:      # near-cancelling: n S_ab - S_a S_b = -(prod mod n) + k n
                s_ab[i, j] = prod // n + (j % 5) - 2
            else:          # correlated sums: S_ab above the product of the means
                s_ab[i, j] = min(prod // n + int(rng.integers(0, 1 << 40)), (1 << 62))
    assert int(s_a[0]) * int(s_b[0]) >= 1 << 63
    dev = "cuda"
    g = torch.empty((ma, mb), dtype=torch.float64, device=dev)
    g32 = torch.empty((mb, ma), dtype=torch.float32, device=dev)
    cpi.cpi_correlate_finalize(torch.from_numpy(s_ab).to(dev), torch.from_numpy(s_a).to(dev),
                               torch.from_numpy(s_b).to(dev), ma, mb, n, g, g32)
    torch.cuda.synchronize()
    want = _expected_bigint(s_ab, s_a, s_b, n)
    got = g.cpu().numpy()
    bad = np.argwhere(got.view(np.int64) != want.view(np.int64))
    assert len(bad) == 0, (len(bad), bad[:3], got[tuple(bad[0])], want[tuple(bad[0])])
    assert np.array_equal(g32.cpu().numpy(), want.astype(np.float32).T)


def test_finalize_wide_numerator_rounding_ties():
    """Numerators in [2^63, 2^64), beyond int64, where doubles are 2^11 apart:
    n = 1, S_a = +-1, S_b = -(2^62 + 2^61), S_ab = +-(2^62 + r), so
    num = +-(2^63 + 2^61 + r); r on, just below and just above a rounding tie
    (2^10 with an even mantissa below, 3 * 2^10 with an odd one), both signs;
    plus n = 3 with a numerator near 2^70 formed by S_a S_b alone."""
    rs = [0, 1, 1023, 1024, 1025, 2047, 2048, 3071, 3072, 3073]
    rows = [(1, 1 << 62 | r) for r in rs] + [(-1, -((1 << 62) + r)) for r in rs]
    ma = len(rows)
    s_a = np.array([a for a, _ in rows], dtype=np.int64)
    s_ab = np.array([[v] for _, v in rows], dtype=np.int64)
    s_b = np.array([-((1 << 62) + (1 << 61))], dtype=np.int64)
    dev = "cuda"
    g = torch.empty((ma, 1), dtype=torch.float64, device=dev)
    cpi.cpi_correlate_finalize(torch.from_numpy(s_ab).to(dev), torch.from_numpy(s_a).to(dev),
                               torch.from_numpy(s_b).to(dev), ma, 1, 1, g, None)
    torch.cuda.synchronize()
    want = _expected_bigint(s_ab, s_a, s_b, 1)
    assert np.array_equal(g.cpu().numpy().view(np.int64), want.view(np.int64))
    assert want[3, 0] == float(2 ** 63 + 2 ** 61) and want[8, 0] == float(2 ** 63 + 2 ** 61 + 4096)
    s_a3 = np.array([(1 << 40) + 1, -((1 << 41) + 7)], dtype=np.int64)
    s_b3 = np.array([-((1 << 30) + 3), (1 << 29) + 5], dtype=np.int64)
    s_ab3 = np.array([[0, 12345], [-99, 1 << 40]], dtype=np.int64)
    g3 = torch.empty((2, 2), dtype=torch.float64, device=dev)
    cpi.cpi_correlate_finalize(torch.from_numpy(s_ab3).to(dev), torch.from_numpy(s_a3).to(dev),
                               torch.from_numpy(s_b3).to(dev), 2, 2, 3, g3, None)
    torch.cuda.synchronize()
    assert np.array_equal(g3.cpu().numpy().view(np.int64), _expected_bigint(s_ab3, s_a3, s_b3, 3).view(np.int64))
