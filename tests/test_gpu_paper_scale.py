"""Paper-scale correlation (Section 2 data layout, Section 4.1 "blocks"): two
256 x 256 binary images side by side in 256 x 512 frames, streamed in blocks of
files (64 files of 512 frames, then a ragged block) through
cpi_correlate_accumulate, then cpi_correlate_finalize: Gamma has 65536 x 65536
entries (34 GB in FP64).  The sums and Gamma must equal the oracle bit for bit
on a sampled band of rows, and the marginal sums everywhere."""

import numpy as np
import pytest
import torch

import paper_2407_20692_gb300 as cpi
import synth
from gpu_util import desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready, oracle_mod):
    yield


def test_256x256_blocks_of_files_accumulate_exactly(oracle_mod):
    blocks = [32768, 32768, 100]
    n = sum(blocks)
    fr = synth.bin_file_frames(n, 2407, device="cuda")
    lay = synth.bin_file_layout()
    ma = mb = 256 * 256
    s_ab = torch.zeros((ma, mb), dtype=torch.int64, device="cuda")
    s_a = torch.zeros(ma, dtype=torch.int64, device="cuda")
    s_b = torch.zeros(mb, dtype=torch.int64, device="cuda")
    ws = torch.empty(cpi.cpi_correlate_workspace_size(desc(fr, lay["a"]), desc(fr, lay["b"]), max(blocks)),
                     dtype=torch.uint8, device="cuda")
    f0 = 0
    for nb in blocks:
        blk = fr[f0:f0 + nb]
        cpi.cpi_correlate_accumulate(desc(blk, lay["a"]), desc(blk, lay["b"]), nb, s_ab, s_a, s_b, ws)
        f0 += nb
    del ws
    gamma = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    cpi.cpi_correlate_finalize(s_ab, s_a, s_b, ma, mb, n, gamma, None)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    r0, r1 = 40000, 40004
    got_sab = s_ab[r0:r1].cpu().numpy()
    got_g = gamma[r0:r1].cpu().numpy()
    got_sa, got_sb = s_a.cpu().numpy(), s_b.cpu().numpy()
    del s_ab, gamma
    host = fr.cpu().numpy()
    del fr
    want = oracle_mod.correlate_rows(host, lay["a"], host, lay["b"], n, r0, r1)
    assert np.array_equal(got_sa, want["s_a"]) and np.array_equal(got_sb, want["s_b"])
    assert np.array_equal(got_sab, want["s_ab"])
    assert np.array_equal(got_g.view(np.int64), want["gamma"].view(np.int64))
