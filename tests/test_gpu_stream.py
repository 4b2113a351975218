"""Streamed acquisitions (cpi_acq_*): frames pushed block by block from host
memory while earlier blocks are accumulated, Gamma finalised mid-stream and at
the end, a checkpoint of the running sums and a resumed acquisition, all
against the oracle on the same frames (sums and Gamma bit for bit) and against
one cpi_correlate call over all frames."""

import numpy as np
import pytest
import torch

import paper_2407_20692_gb300 as cpi
import synth
from gpu_util import assert_exact, desc, gpu_correlate, oracle_correlate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready, oracle_mod):
    yield


def _outputs(ma, mb):
    z = lambda *s: torch.empty(s, dtype=torch.int64, device="cuda")
    return z(ma, mb), z(ma), z(mb)


@pytest.mark.parametrize("counts,sa,sb,n,block", [("bernoulli", 64, 32, 9000, 2048),
                                                 ("poisson8", 40, 24, 5000, 1536),
                                                 ("bernoulli", 24, 16, 700, 700)])
def test_streamed_acquisition_matches_oracle_and_single_call(counts, sa, sb, n, block):
    acq = synth.Acquisition(sa, sb, n, 0.3 if counts == "bernoulli" else 2.0, counts, seed=77)
    A, B = synth.generate(acq, "cuda")
    fr, lay = synth.pack_side_by_side(A, B, acq.bits)
    host = fr.cpu().pin_memory()
    a, b = desc(fr, lay["a"]), desc(fr, lay["b"])
    ma, mb = sa * sa, sb * sb
    s_ab, s_a, s_b = _outputs(ma, mb)
    ws = torch.empty(cpi.cpi_acq_workspace_size(a, b, block), dtype=torch.uint8, device="cuda")
    h = cpi.cpi_acq_begin(a, b, block, s_ab, s_a, s_b, ws)
    half = (n // 2) // block * block or block
    g_mid = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    pushed = 0
    while pushed < n:
        k = min(block, n - pushed)
        cpi.cpi_acq_push(h, host[pushed:pushed + k], k)
        pushed += k
        if pushed == half:
            cpi.cpi_acq_finalize(h, g_mid, None)      # Gamma of the first half, acquisition goes on
    assert cpi.cpi_acq_frames(h) == n
    g = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    g32 = torch.empty((mb, ma), dtype=torch.float32, device="cuda")
    cpi.cpi_acq_finalize(h, g, g32)
    cpi.cpi_acq_end(h)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    hn = fr.cpu().numpy()
    want = oracle_correlate(hn, lay["a"], lay["b"], n)
    assert_exact({"s_ab": s_ab.cpu(), "s_a": s_a.cpu(), "s_b": s_b.cpu(), "gamma": g.cpu()}, want)
    want_half = oracle_correlate(hn, lay["a"], lay["b"], half)
    assert np.array_equal(g_mid.cpu().numpy().view(np.int64), want_half["gamma"].view(np.int64))
    one = gpu_correlate(fr, lay["a"], lay["b"], n)
    assert torch.equal(one["gamma_f32"].cpu(), g32.cpu())


def test_checkpoint_and_resume():
    """Sums saved after cpi_acq_sync are the complete state: a new acquisition
    begun from them (frames_done > 0) continues to the same Gamma."""
    acq = synth.Acquisition(32, 16, 6000, 0.3, "bernoulli", seed=91)
    A, B = synth.generate(acq, "cuda")
    fr, lay = synth.pack_side_by_side(A, B, 1)
    host = fr.cpu().pin_memory()
    a, b = desc(fr, lay["a"]), desc(fr, lay["b"])
    ma, mb, block = 1024, 256, 1000
    s_ab, s_a, s_b = _outputs(ma, mb)
    ws = torch.empty(cpi.cpi_acq_workspace_size(a, b, block), dtype=torch.uint8, device="cuda")
    h = cpi.cpi_acq_begin(a, b, block, s_ab, s_a, s_b, ws)
    for f0 in range(0, 3000, block):
        cpi.cpi_acq_push(h, host[f0:f0 + block], block)
    cpi.cpi_acq_sync(h)
    saved = [t.clone() for t in (s_ab, s_a, s_b)]          # checkpoint
    cpi.cpi_acq_end(h)
    r_ab, r_a, r_b = [t.clone() for t in saved]
    h = cpi.cpi_acq_begin(a, b, block, r_ab, r_a, r_b, ws, frames_done=3000)
    for f0 in range(3000, 6000, block):
        cpi.cpi_acq_push(h, host[f0:f0 + block], block)
    g = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    cpi.cpi_acq_finalize(h, g, None)
    cpi.cpi_acq_end(h)
    torch.cuda.synchronize()
    want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], 6000)
    assert_exact({"s_ab": r_ab.cpu(), "s_a": r_a.cpu(), "s_b": r_b.cpu(), "gamma": g.cpu()}, want)


def test_binary_blocks_of_mixed_sizes():
    """Binary acquisitions keep the raw moments of full blocks in the workspace's
    uint32 partial slots and fold them into S_ab at a checkpoint or before a
    block of another size: full, full, short, full, full, then Gamma, against the
    oracle bit for bit."""
    sizes = [1024, 1024, 300, 1024, 1024]
    n = sum(sizes)
    acq = synth.Acquisition(48, 24, n, 0.3, "bernoulli", seed=123)
    A, B = synth.generate(acq, "cuda")
    fr, lay = synth.pack_side_by_side(A, B, 1)
    host = fr.cpu().pin_memory()
    a, b = desc(fr, lay["a"]), desc(fr, lay["b"])
    ma, mb = 48 * 48, 24 * 24
    s_ab, s_a, s_b = _outputs(ma, mb)
    ws = torch.empty(cpi.cpi_acq_workspace_size(a, b, 1024), dtype=torch.uint8, device="cuda")
    h = cpi.cpi_acq_begin(a, b, 1024, s_ab, s_a, s_b, ws)
    f0 = 0
    for k in sizes:
        cpi.cpi_acq_push(h, host[f0:f0 + k], k)
        f0 += k
    g = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    cpi.cpi_acq_finalize(h, g, None)
    cpi.cpi_acq_end(h)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], n)
    assert_exact({"s_ab": s_ab.cpu(), "s_a": s_a.cpu(), "s_b": s_b.cpu(), "gamma": g.cpu()}, want)


def test_acquisition_argument_errors():
    fr = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    a = cpi.frames(fr, 1, 8, 8, 0, 0, 16, 16)
    b = cpi.frames(fr, 1, 8, 8, 8, 0, 16, 16)
    bad = cpi.frames(fr, 1, 8, 8, 8, 0, 16, 32)              # another frame stride
    assert cpi.cpi_acq_workspace_size(a, bad, 100) == 0
    assert cpi.cpi_acq_workspace_size(a, b, 0) == 0
    s_ab, s_a, s_b = _outputs(64, 64)
    ws = torch.empty(cpi.cpi_acq_workspace_size(a, b, 100), dtype=torch.uint8, device="cuda")
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_acq_begin(a, b, 100, s_ab, s_a, s_b, ws[:64])
    assert e.value.code == 3
    h = cpi.cpi_acq_begin(a, b, 100, s_ab, s_a, s_b, ws)
    host = torch.zeros(200 * 16, dtype=torch.uint8).pin_memory()
    with pytest.raises(cpi.CpiError) as e:                   # more frames than a block holds
        cpi.cpi_acq_push(h, host, 101)
    assert e.value.code == 1
    with pytest.raises(cpi.CpiError) as e:                   # nothing pushed yet
        cpi.cpi_acq_finalize(h, torch.empty((64, 64), dtype=torch.float64, device="cuda"), None)
    assert e.value.code == 1
    cpi.cpi_acq_end(h)
