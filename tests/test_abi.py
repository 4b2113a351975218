"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/cpi.h declares; host-side planning answers without a device."""

import ctypes
import os
import re

import pytest

import paper_2407_20692_gb300 as cpi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cpi.h")).read()
    return sorted(set(re.findall(r"^CPI_API[^(]*?\b(cpi_\w+)\(", src, flags=re.M)))


def test_header_declares_the_binding_names():
    assert _declared() == sorted(cpi.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = cpi.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert cpi.cpi_abi_version() == 1
    assert cpi.cpi_status_string(0) == "CPI_OK"
    assert cpi.cpi_status_string(6) == "CPI_ERR_TIMEOUT"


def test_library_has_no_cpu_fallback_symbols():
    """The product library contains no oracle code."""
    data = open(cpi.library_path(), "rb").read()
    assert b"oracle_correlate" not in data and b"oracle_refocus" not in data


def _fd(bits, h, w, x0=0, rs=None, fs=None):
    rs = rs or (x0 + w)
    fs = fs or (h * rs if bits == 8 else (h * rs + 7) // 8)
    return cpi.cpi_frames(0x1000, bits, h, w, x0, 0, rs, fs, 0)


def test_workspace_query_host_logic():
    # binary 64x64 vs 32x32, 20000 frames: E2M1 operands (two frames per byte)
    # padded to 256 frames, plus the uint32 partial sums
    a, b = _fd(1, 64, 64, 0, 96), _fd(1, 32, 32, 64, 96, 64 * 96 // 8)
    a.frame_stride_bytes = 64 * 96 // 8
    ws = cpi.cpi_correlate_workspace_size(a, b, 20000)
    kpad = 20224
    need = (4096 + 1024) * kpad // 2 + 4096 * 1024 * 4
    assert need <= ws < need + 64 * 1024
    # uint8 inputs use BF16 operands (2 bytes per frame)
    a8, b8 = _fd(8, 16, 16), _fd(8, 16, 16)
    ws8 = cpi.cpi_correlate_workspace_size(a8, b8, 2000)
    assert ws8 >= (256 + 256) * 2048 * 2 + 256 * 256 * 4
    # invalid descriptors and sizes answer 0
    assert cpi.cpi_correlate_workspace_size(a8, b8, 0) == 0
    bad = _fd(8, 16, 16)
    bad.bits = 3
    assert cpi.cpi_correlate_workspace_size(bad, b8, 10) == 0
    outside = _fd(8, 16, 16)
    outside.frame_stride_bytes = 100          # region does not fit in one frame
    assert cpi.cpi_correlate_workspace_size(outside, b8, 10) == 0
    assert cpi.cpi_refocus_workspace_size(64, 64, 32, 32, 32) > 0
    assert cpi.cpi_refocus_workspace_size(0, 64, 32, 32, 32) == 0


def test_refocus_workspace_layout():
    """The x stage's images [planes][hb][ha][wa] for up to 128 planes (larger
    stacks run in chunks of 128 that reuse them), then, when Gamma's rows do not
    meet the staging alignment, a copy of Gamma with padded rows: to a multiple
    of 4 floats for rows up to 248 wide (2-D staging), of 16 floats above
    (3-D staging in 16-float chunks); last the fixed-point x-coordinate tables
    of one launch (128 planes x 512 column threads, and two values per plane)."""
    up = lambda n: -(-n // 256) * 256
    for ha, wa, hb, wb, P in [(33, 70, 7, 5, 7), (46, 95, 4, 4, 3), (17, 33, 5, 3, 2), (64, 64, 32, 32, 32),
                              (128, 128, 64, 64, 128), (12, 10, 3, 4, 200), (5, 300, 3, 2, 7), (9, 256, 2, 2, 3),
                              (256, 256, 4, 4, 100), (3, 512, 2, 2, 2), (4, 249, 2, 2, 1)]:
        ws = cpi.cpi_refocus_workspace_size(ha, wa, hb, wb, P)
        want = up(min(P, 128) * hb * ha * wa * 4)
        pitch = (wa + 3) // 4 * 4 if wa <= 248 else (wa + 15) // 16 * 16
        if pitch != wa:
            want += up(hb * wb * ha * pitch * 4)
        want += up(128 * 512 * 8) + up(128 * 2 * 8)      # fixed-point x-coordinate tables of one launch
        assert ws == want, (ha, wa, hb, wb, P, ws, want)
    # rows wider than 512 are refused (0)
    assert cpi.cpi_refocus_workspace_size(4, 513, 2, 2, 1) == 0


def test_denoise_workspace_has_channels_last_buffers_for_tensor_core_widths():
    """Inference layout: scale, sums, x (9 channels), a1..a3 (32 channels, bf16),
    y (float), each rounded up to 256 bytes; widths 32, 64 and 128 (the
    tensor-core layers) add three channels-last copies of 64 bytes per pixel and
    the bf16 weights of the four layers."""
    up = lambda n: -(-n // 256) * 256
    for ha, wa, hb, wb in [(16, 32, 4, 4), (8, 64, 2, 3), (5, 128, 2, 2), (16, 40, 4, 4), (12, 20, 3, 4)]:
        B, HW = hb * wb, ha * wa
        want = up(4) + up(8 * 256) + up(2 * B * 9 * HW) + 3 * up(2 * B * 32 * HW) + up(4 * B * HW)
        if wa in (32, 64, 128):
            want += 3 * up(64 * B * HW) + up(2 * (3 * 9 * 32 * 32 + 9 * 16 * 32))
        assert cpi.cpi_denoise_workspace_size(ha, wa, hb, wb) == want, (ha, wa, hb, wb)
        # training adds dy, two float32 gradient buffers of 32 channels and the
        # per-CTA partials; width 64 (tensor-core weight gradients) also the
        # split gradient (64 bf16 channels), the shifted input copies (96 bf16
        # channels), the GEMM partials (304 x 64 x 288 floats), the bias sums, the
        # channels-last split gradient and the flipped weights of the input gradients
        want += up(4 * B * HW) + 2 * up(4 * B * 32 * HW) + up(4 * 456 * (32 * 32 * 9 + 32))
        if wa == 64:
            want += up(2 * B * 64 * HW) + up(2 * B * 96 * HW) + up(4 * 304 * 64 * 288)
            want += up(4 * B * (-(-HW // 256)) * 32)                       # bias sums per (slice, 256 pixels)
            want += 2 * up(2 * B * 32 * HW) + up(2 * 2 * 9 * 32 * 32)      # channels-last split, flipped weights
        assert cpi.cpi_denoise_workspace_size(ha, wa, hb, wb, training=True) == want, (ha, wa, hb, wb)


def test_refocus4d_workspace_chunks_planes():
    """Up to 64 planes per chunk, fewer when a chunk's column sums would pass 4 GB."""
    small = cpi.cpi_refocus4d_workspace_size(16, 16, 8, 8, 10)
    more = cpi.cpi_refocus4d_workspace_size(16, 16, 8, 8, 500)
    assert 0 < small < more
    assert more == cpi.cpi_refocus4d_workspace_size(16, 16, 8, 8, 64)   # one 64-plane chunk is reused
    big = cpi.cpi_refocus4d_workspace_size(256, 256, 256, 256, 100)
    assert big <= (4 << 30) + (1 << 24)
