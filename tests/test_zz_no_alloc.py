"""cpi_correlate_noalloc: Eq. (1) with the library's built-in scratch.

Some callers cannot allocate device memory -- a real-time acquisition loop that
cannot afford cudaMalloc's device synchronisation, or a host application whose
own allocator owns all device memory.  For them the library offers one entry
point that takes inputs and outputs only and works in a fixed scratch array the
library keeps on each GPU.  Its results must equal those of cpi_correlate (which
works in a caller-provided workspace) bit for bit, call after call, although
every call reuses the same array.  This file is collected last so that a run
stopping at the first failure has already run every other test."""

import numpy as np
import pytest
import torch

import paper_2407_20692_gb300 as cpi
import synth
from gpu_util import desc, make_frames

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready):
    yield


def _outputs(ma, mb):
    dev = "cuda"
    return (torch.empty((ma, mb), dtype=torch.int64, device=dev),
            torch.empty(ma, dtype=torch.int64, device=dev),
            torch.empty(mb, dtype=torch.int64, device=dev),
            torch.empty((ma, mb), dtype=torch.float64, device=dev),
            torch.empty((mb, ma), dtype=torch.float32, device=dev))


def _both(acq):
    fr, lay = make_frames(acq)
    a, b = desc(fr, lay["a"]), desc(fr, lay["b"])
    n = acq.n_frames
    ma = lay["a"]["height"] * lay["a"]["width"]
    mb = lay["b"]["height"] * lay["b"]["width"]
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, n), dtype=torch.uint8, device="cuda")
    assert ws.numel() <= cpi.NOALLOC_SCRATCH_BYTES
    ref = _outputs(ma, mb)
    cpi.cpi_correlate(a, b, n, *ref, ws)
    got = _outputs(ma, mb)
    cpi.cpi_correlate_noalloc(a, b, n, *got)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    return ref, got


def test_noalloc_equals_workspace_entry_point_on_consecutive_calls():
    # two calls in a row on different acquisitions (binary, then uint8 counts):
    # the second call must not see anything the first one left in the scratch
    for acq in (synth.Acquisition(24, 12, 3001, 0.3, "bernoulli", seed=11),
                synth.Acquisition(16, 16, 2000, 2.0, "poisson8", seed=12),
                synth.Acquisition(24, 12, 1500, 0.3, "bernoulli", seed=13)):
        ref, got = _both(acq)
        for r, g in zip(ref, got):
            assert torch.equal(r.cpu(), g.cpu())
        # Gamma bit for bit (same exact numerator, same rounding)
        assert np.array_equal(ref[3].cpu().numpy().view(np.int64), got[3].cpu().numpy().view(np.int64))


def test_noalloc_refuses_problems_larger_than_its_scratch():
    acq = synth.CONFIGS["spad_1bit"]     # 16384 frames: ~60 MB of workspace
    fr, lay = make_frames(acq, n=16384)
    a, b = desc(fr, lay["a"]), desc(fr, lay["b"])
    assert cpi.cpi_correlate_workspace_size(a, b, 16384) > cpi.NOALLOC_SCRATCH_BYTES
    out = _outputs(4096, 1024)
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_correlate_noalloc(a, b, 16384, *out)
    assert e.value.code == 3
