"""GPU parity of Eq. (1): the CUDA path through the C ABI against the CPU oracle.

S_ab, S_a, S_b must be bit-exact and Gamma bit-identical (same exact int64
numerator, one correctly rounded conversion and division on both sides)."""

import json
import os

import numpy as np
import pytest
import torch

import paper_2407_20692_gb300 as cpi
import synth
from gpu_util import assert_exact, desc, gpu_correlate, make_frames, oracle_correlate

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready, oracle_mod):
    yield


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "eq1_hand.json")))["cases"],
                         ids=lambda c: c["name"])
def test_hand_worked_cases(case):
    fr = torch.tensor(case["frames"], dtype=torch.uint8, device="cuda")
    common = dict(bits=case["bits"], row_stride=case["row_stride"],
                  frame_stride_bytes=case["frame_stride_bytes"], bit_order=case["bit_order"])
    la, lb = dict(common, **case["a"]), dict(common, **case["b"])
    got = gpu_correlate(fr, la, lb, len(case["frames"]))
    assert got["s_ab"].tolist() == case["s_ab"]
    assert got["s_a"].tolist() == case["s_a"]
    from fractions import Fraction

    want = np.array([[float(Fraction(x)) for x in row] for row in case["gamma"]])
    assert np.array_equal(got["gamma"].numpy(), want)


@pytest.mark.parametrize("side_a,side_b,n,counts", [
    (16, 16, 2000, "poisson8"),          # the small 16x16 vs 16x16 uint8 workload, full size
    (24, 12, 3001, "bernoulli"),         # ragged tiles and a ragged frame count
    (20, 9, 777, "poisson8"),            # rows not 4-byte aligned: the per-byte ingest
    (36, 20, 1234, "poisson8"),          # 4-pixel ingest: ragged 128-pixel tiles and frame tail
    (40, 36, 4500, "bernoulli"),         # several M and N tiles, N tile ragged
    (8, 40, 300, "binomial255"),         # M_a < one tile, large counts
])
def test_correlate_matches_oracle(side_a, side_b, n, counts):
    acq = synth.Acquisition(side_a, side_b, n, 2.0 if counts == "poisson8" else 0.3, counts, seed=7)
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], n)
    want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], n)
    assert_exact(got, want)


def test_correlate_spad_1bit_full_size():
    """64x64 vs 32x32 binary frames, 20000 frames, bit-packed side by side."""
    acq = synth.CONFIGS["spad_1bit"]
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], acq.n_frames)
    want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], acq.n_frames)
    assert_exact(got, want)


def test_correlate_large_u8_sampled_rows():
    """128x128 vs 64x64 uint8 (sums of 255 binary sub-frames), 50000 frames:
    two frame chunks; full S_a, S_b and sampled row blocks of S_ab / Gamma."""
    acq = synth.CONFIGS["large_u8"]
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], acq.n_frames, want_f32=False)
    host = fr.cpu().numpy()
    del fr
    torch.cuda.empty_cache()
    for rows in [(0, 24), (8100, 8140), (16384 - 16, 16384)]:
        want = oracle_correlate(host, lay["a"], lay["b"], acq.n_frames, rows=rows)
        assert_exact(got, want, rows=rows)


def test_exactness_adversarial_all_ones_and_max_counts():
    """Partial sums at the exactness bounds on a small output (whose frames are
    split into many chunks to fill the GPU, then added by the fold): all-ones
    binary frames, and all-255 counts (products 65025) over 33000 frames."""
    n = 32768 + 300
    ha, wa, hb, wb = 4, 8, 2, 8
    W = wa + wb
    img = torch.ones((n, ha, W), dtype=torch.uint8)
    bits = synth.pack_bits_lsb(img.reshape(n, ha * W))
    fr = bits.cuda()
    la = dict(bits=1, height=ha, width=wa, x0=0, y0=0, row_stride=W, frame_stride_bytes=ha * W // 8)
    lb = dict(la, height=hb, width=wb, x0=wa)
    got = gpu_correlate(fr, la, lb, n)
    assert (got["s_ab"] == n).all() and (got["s_a"] == n).all() and (got["s_b"] == n).all()
    assert (got["gamma"] == 0).all()
    n2 = 33000
    fr8 = torch.full((n2, ha * W), 255, dtype=torch.uint8, device="cuda")
    fr8[::3, 0] = 254        # break the symmetry a little
    l8a = dict(bits=8, height=ha, width=wa, x0=0, y0=0, row_stride=W, frame_stride_bytes=ha * W)
    l8b = dict(l8a, height=hb, width=wb, x0=wa)
    got = gpu_correlate(fr8, l8a, l8b, n2)
    want = oracle_correlate(fr8.cpu().numpy(), l8a, l8b, n2)
    assert_exact(got, want)


@pytest.mark.parametrize("n", [65536, 65600])
def test_full_chunk_of_max_counts_closed_form(n):
    """A frame chunk holds up to 65536 frames: with counts of 255 every partial
    sum passes 2^31 (65536 x 255^2 = 4.26e9 < 2^32, kept as uint32).  2560 x 2048
    outputs (160 tiles, so no extra frame split): n = 65536 is one chunk, finished
    in the raw-moment epilogue; n = 65600 is two chunks, added by the fold.
    A_i[a] = 255 - [a == 0][i % 3 == 0], B_i[b] = 255 - [b == 0][i % 5 == 0];
    the sums follow by counting frames, Gamma from Python big integers."""
    ha, wa, hb, wb = 40, 64, 32, 64
    W = wa + wb
    fr = torch.full((n, ha, W), 255, dtype=torch.uint8, device="cuda")
    i = torch.arange(n, device="cuda")
    fr[i % 3 == 0, 0, 0] = 254
    fr[i % 5 == 0, 0, wa] = 254
    la = dict(bits=8, height=ha, width=wa, x0=0, y0=0, row_stride=W, frame_stride_bytes=ha * W)
    lb = dict(la, height=hb, width=wb, x0=wa)
    got = gpu_correlate(fr, la, lb, n, want_f32=False)
    ma, mb = ha * wa, hb * wb
    c3, c5, c15 = (n + 2) // 3, (n + 4) // 5, (n + 14) // 15
    sa = np.full(ma, 255 * n, dtype=np.int64)
    sa[0] -= c3
    sb = np.full(mb, 255 * n, dtype=np.int64)
    sb[0] -= c5
    sab = np.full((ma, mb), 255 * 255 * n, dtype=np.int64)
    sab[0, :] -= 255 * c3
    sab[:, 0] -= 255 * c5
    sab[0, 0] += c15
    assert np.array_equal(got["s_a"].numpy(), sa) and np.array_equal(got["s_b"].numpy(), sb)
    assert np.array_equal(got["s_ab"].numpy(), sab)
    assert int(sab.max()) > 2 ** 31
    g = got["gamma"].numpy()
    d = float(n) * float(n)
    for (a, b) in [(0, 0), (0, 1), (1, 0), (1, 1), (ma - 1, mb - 1)]:
        want = float(n * int(sab[a, b]) - int(sa[a]) * int(sb[b])) / d
        assert g[a, b] == want, (a, b, g[a, b], want)
    assert (g[1:, 1:] == 0.0).all()


@pytest.mark.parametrize("top", [23, 91, 255])
def test_segment_length_follows_the_recorded_value_range(top):
    """8-bit frames: the FP32 tensor-memory accumulator is folded into uint32
    every S frames, S the largest multiple of 64 with S x max A x max B < 2^24
    (from the maxima the ingest records; at top = 255 the segment sums reach
    16,646,400, within 2 frames' worth of 2^24).  Constant A = top and B = top
    except in every 16th frame (top - 1) make every tensor-core K step add an
    odd increment, so a segment that overran 2^24 (where FP32 integers are 2
    apart) would lose low bits and the sums would be wrong.  2048 x 1280 outputs
    keep the 32768 frames in one chunk (several segments per unit for every top)."""
    n = 32768
    ha, wa, hb, wb = 32, 64, 20, 64
    W = wa + wb
    fr = torch.full((n, ha, W), top, dtype=torch.uint8, device="cuda")
    low = torch.arange(n, device="cuda") % 16 == 0
    fr[low, :hb, wa:] = top - 1
    la = dict(bits=8, height=ha, width=wa, x0=0, y0=0, row_stride=W, frame_stride_bytes=ha * W)
    lb = dict(la, height=hb, width=wb, x0=wa)
    got = gpu_correlate(fr, la, lb, n)
    n_low = int(low.sum().item())
    assert (got["s_a"] == top * n).all()
    assert (got["s_b"] == top * n - n_low).all()
    assert (got["s_ab"] == top * (top * n - n_low)).all()


def test_mixed_bit_depths():
    """A binary, B uint8 from different buffers."""
    acq = synth.Acquisition(20, 10, 2500, 1.0, "poisson8", seed=3)
    A, B = synth.generate(acq, "cuda")
    Ab = (A > 0).to(torch.uint8)
    fa, la = synth.pack_side_by_side(Ab, torch.zeros((acq.n_frames, 1, 1), dtype=torch.uint8, device="cuda"), 1)
    fb = B.reshape(acq.n_frames, -1).contiguous()
    lb = dict(bits=8, height=10, width=10, x0=0, y0=0, row_stride=10, frame_stride_bytes=100)
    a, b = desc(fa, la["a"]), desc(fb, lb)
    n = acq.n_frames
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, n), dtype=torch.uint8, device="cuda")
    s_ab = torch.empty((400, 100), dtype=torch.int64, device="cuda")
    s_a = torch.empty(400, dtype=torch.int64, device="cuda")
    s_b = torch.empty(100, dtype=torch.int64, device="cuda")
    g = torch.empty((400, 100), dtype=torch.float64, device="cuda")
    cpi.cpi_correlate(a, b, n, s_ab, s_a, s_b, g, None, ws)
    torch.cuda.synchronize()
    import oracle

    want = oracle.correlate(fa.cpu().numpy(), la["a"], fb.cpu().numpy(), lb, n)
    assert np.array_equal(s_ab.cpu().numpy(), want["s_ab"])
    assert np.array_equal(g.cpu().numpy().view(np.int64), want["gamma"].view(np.int64))


def test_accumulate_then_finalize_equals_single_call():
    acq = synth.Acquisition(32, 16, 6000, 0.3, "bernoulli", seed=5)
    fr, lay = make_frames(acq)
    n = acq.n_frames
    full = gpu_correlate(fr, lay["a"], lay["b"], n)
    a1, b1 = desc(fr, lay["a"]), desc(fr, lay["b"])
    ma, mb = 32 * 32, 16 * 16
    s_ab = torch.zeros((ma, mb), dtype=torch.int64, device="cuda")
    s_a = torch.zeros(ma, dtype=torch.int64, device="cuda")
    s_b = torch.zeros(mb, dtype=torch.int64, device="cuda")
    fb = lay["frame_bytes"]
    for f0, f1 in [(0, 2500), (2500, 2501), (2501, 6000)]:
        sub = fr[f0:f1]
        a, b = desc(sub, lay["a"]), desc(sub, lay["b"])
        ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, f1 - f0), dtype=torch.uint8, device="cuda")
        cpi.cpi_correlate_accumulate(a, b, f1 - f0, s_ab, s_a, s_b, ws)
    g = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    g32 = torch.empty((mb, ma), dtype=torch.float32, device="cuda")
    cpi.cpi_correlate_finalize(s_ab, s_a, s_b, ma, mb, n, g, g32)
    torch.cuda.synchronize()
    assert torch.equal(s_ab.cpu(), full["s_ab"])
    assert torch.equal(g.cpu(), full["gamma"])
    assert torch.equal(g32, full["gamma_f32"])
    assert fb > 0


def test_stages_equal_single_call():
    acq = synth.Acquisition(48, 24, 3000, 0.3, "bernoulli", seed=9)
    fr, lay = make_frames(acq)
    n = acq.n_frames
    full = gpu_correlate(fr, lay["a"], lay["b"], n)
    a, b = desc(fr, lay["a"]), desc(fr, lay["b"])
    ma, mb = 48 * 48, 24 * 24
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, n), dtype=torch.uint8, device="cuda")
    s_ab = torch.empty((ma, mb), dtype=torch.int64, device="cuda")
    s_a = torch.empty(ma, dtype=torch.int64, device="cuda")
    s_b = torch.empty(mb, dtype=torch.int64, device="cuda")
    g = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    for st in (cpi.CPI_STAGE_INGEST, cpi.CPI_STAGE_MOMENTS, cpi.CPI_STAGE_FOLD):
        cpi.cpi_correlate_stage(st, a, b, n, 0, s_ab, s_a, s_b, g, None, ws)
    torch.cuda.synchronize()
    assert torch.equal(s_ab.cpu(), full["s_ab"])
    assert torch.equal(g.cpu(), full["gamma"])


def test_gamma_f32_is_slice_major_copy():
    acq = synth.Acquisition(24, 12, 1000, 2.0, "poisson8", seed=2)
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], acq.n_frames)
    assert torch.equal(got["gamma_f32"].cpu(), got["gamma"].float().T.contiguous())


def test_same_detector_symmetric():
    acq = synth.Acquisition(16, 16, 4000, 0.3, "bernoulli", seed=4)
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["a"], acq.n_frames)
    g = got["gamma"]
    assert torch.equal(g, g.T)


def test_argument_errors_are_reported_before_launch():
    fr = torch.zeros(64, dtype=torch.uint8, device="cuda")
    good = dict(bits=1, height=4, width=4, x0=0, y0=0, row_stride=8, frame_stride_bytes=4)
    a = desc(fr, good)
    s = torch.zeros((16, 16), dtype=torch.int64, device="cuda")
    v = torch.zeros(16, dtype=torch.int64, device="cuda")
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, a, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_correlate(a, a, 0, s, v, v, None, None, ws)
    assert e.value.code == 1
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_correlate(a, a, 16, s, v, v, None, None, ws[:16])
    assert e.value.code == 3
    bad = desc(fr, dict(good, bits=4))
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_correlate(bad, a, 16, s, v, v, None, None, ws)
    assert e.value.code == 1
    big8 = desc(fr, dict(good, bits=8, frame_stride_bytes=32))
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_correlate(big8, big8, 20_000_000, s, v, v, None, None, ws)
    assert e.value.code == 2
    with pytest.raises(cpi.CpiError) as e:       # missing model and Gamma buffers
        cpi.cpi_denoise(None, None, None, 4, 4, 4, 4, ws)
    assert e.value.code == 1
    g = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    for stage in (cpi.CPI_STAGE_INGEST, cpi.CPI_STAGE_MOMENTS, cpi.CPI_STAGE_FOLD):
        # an accumulating call has no total frame count: it must not write Gamma
        with pytest.raises(cpi.CpiError) as e:
            cpi.cpi_correlate_stage(stage, a, a, 16, 1, s, v, v, g, None, ws)
        assert e.value.code == 1


def test_wait_timeout_is_reported_and_context_survives():
    """A barrier wait that nothing satisfies gives up after its limit; the status
    word reports CPI_ERR_TIMEOUT and later work still runs."""
    assert cpi.cpi_device_status() == 0
    cpi.cpi_selftest_wait_timeout(50_000_000)          # 50 ms
    assert cpi.cpi_device_status(clear=True) == 6
    assert cpi.cpi_device_status() == 0
    acq = synth.Acquisition(16, 16, 500, 2.0, "poisson8", seed=1)
    fr, lay = make_frames(acq)
    got = gpu_correlate(fr, lay["a"], lay["b"], acq.n_frames)
    want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], acq.n_frames)
    assert_exact(got, want)


@pytest.mark.parametrize("bit_order,xa,xb,wa,wb", [(0, 0, 64, 64, 32), (1, 0, 64, 64, 32),
                                                   (0, 5, 77, 64, 32), (1, 3, 70, 32, 64),
                                                   (0, 1, 40, 37, 20)])
def test_bit_layouts_match_oracle(bit_order, xa, xb, wa, wb):
    """Region origins off word boundaries, MSB-first bytes, widths that are and
    are not multiples of 32 (word-load path and per-pixel path)."""
    rng = np.random.default_rng(bit_order * 100 + xa)
    n, H = 1500, 6
    W = max(xa + wa, xb + wb) + 3
    img = (rng.random((n, H, W)) < 0.35).astype(np.uint8)
    flat = torch.from_numpy(img.reshape(n, H * W))
    pad = (-flat.shape[1]) % 32
    flat = torch.cat([flat, torch.zeros((n, pad), dtype=torch.uint8)], 1)
    packed = synth.pack_bits_lsb(flat)
    if bit_order == 1:
        lut = torch.tensor([int('{:08b}'.format(v)[::-1], 2) for v in range(256)], dtype=torch.uint8)
        packed = lut[packed.long()]
    fs = packed.shape[1]
    fr = packed.contiguous().cuda()
    la = dict(bits=1, height=H, width=wa, x0=xa, y0=0, row_stride=W, frame_stride_bytes=fs, bit_order=bit_order)
    lb = dict(bits=1, height=H - 1, width=wb, x0=xb, y0=1, row_stride=W, frame_stride_bytes=fs, bit_order=bit_order)
    got = gpu_correlate(fr, la, lb, n)
    want = oracle_correlate(fr.cpu().numpy(), la, lb, n)
    assert_exact(got, want)
    A = img[:, 0:H, xa:xa + wa].reshape(n, -1).astype(np.int64)
    assert np.array_equal(got["s_a"].numpy(), A.sum(0))


@pytest.mark.parametrize("bit_order", [0, 1])
def test_bit_regions_spanning_several_word_chunks(bit_order):
    """Binary frames of 40 rows x 203 bits (254 words per frame): both regions
    span several 64-word chunks of the word-staged ingest, with tiles whose two
    words straddle a chunk edge; 700 frames (not a whole frame block)."""
    rng = np.random.default_rng(40 + bit_order)
    n, H, W = 700, 40, 203
    img = (rng.random((n, H, W)) < 0.3).astype(np.uint8)
    flat = torch.from_numpy(img.reshape(n, H * W))
    pad = (-flat.shape[1]) % 32
    flat = torch.cat([flat, torch.zeros((n, pad), dtype=torch.uint8)], 1)
    packed = synth.pack_bits_lsb(flat)
    if bit_order == 1:
        lut = torch.tensor([int('{:08b}'.format(v)[::-1], 2) for v in range(256)], dtype=torch.uint8)
        packed = lut[packed.long()]
    fs = packed.shape[1]
    fr = packed.contiguous().cuda()
    la = dict(bits=1, height=H, width=64, x0=5, y0=0, row_stride=W, frame_stride_bytes=fs, bit_order=bit_order)
    lb = dict(bits=1, height=H - 3, width=96, x0=90, y0=2, row_stride=W, frame_stride_bytes=fs, bit_order=bit_order)
    got = gpu_correlate(fr, la, lb, n)
    want = oracle_correlate(fr.cpu().numpy(), la, lb, n)
    assert_exact(got, want)


@pytest.mark.parametrize("counts", ["bernoulli", "poisson8"])
def test_sums_may_stay_in_the_workspace(counts):
    """Without caller buffers for S_ab, S_a, S_b the marginals live in the
    workspace and S_ab is not written; Gamma (both layouts) is bit-identical to
    the call that returns every sum.  Accumulating calls still need the sums."""
    acq = synth.Acquisition(24, 12, 2500, 2.0 if counts == "poisson8" else 0.4, counts, seed=41)
    fr, lay = make_frames(acq)
    full = gpu_correlate(fr, lay["a"], lay["b"], 2500)
    a, b = desc(fr, lay["a"]), desc(fr, lay["b"])
    ma, mb = 24 * 24, 12 * 12
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, 2500), dtype=torch.uint8, device="cuda")
    g = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    g32 = torch.empty((mb, ma), dtype=torch.float32, device="cuda")
    cpi.cpi_correlate(a, b, 2500, None, None, None, g, g32, ws)
    torch.cuda.synchronize()
    assert torch.equal(g.cpu(), full["gamma"])
    assert torch.equal(g32, full["gamma_f32"])
    with pytest.raises(cpi.CpiError) as e:      # nothing to return
        cpi.cpi_correlate(a, b, 2500, None, None, None, None, None, ws)
    assert e.value.code == 1
    s = torch.zeros((ma, mb), dtype=torch.int64, device="cuda")
    with pytest.raises(cpi.CpiError) as e:      # accumulating into missing sums
        cpi.cpi_correlate_accumulate(a, b, 2500, s, None, None, ws)
    assert e.value.code == 1
