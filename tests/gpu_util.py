"""Shared helpers for the GPU parity tests: run the library on frames and run the
oracle on the same frames."""

import numpy as np
import torch

import paper_2407_20692_gb300 as cpi
import synth


def desc(frames_dev, lay):
    return cpi.frames(frames_dev, lay["bits"], lay["height"], lay["width"], lay["x0"], lay["y0"],
                      lay["row_stride"], lay["frame_stride_bytes"], lay.get("bit_order", 0))


def gpu_correlate(frames_dev, la, lb, n, want_f32=True, stream=None):
    """Eq. (1) on the GPU through the C ABI. Returns dict of CPU tensors."""
    a, b = desc(frames_dev, la), desc(frames_dev, lb)
    ma, mb = la["height"] * la["width"], lb["height"] * lb["width"]
    dev = frames_dev.device
    ws_bytes = cpi.cpi_correlate_workspace_size(a, b, n)
    assert ws_bytes > 0
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    s_ab = torch.empty((ma, mb), dtype=torch.int64, device=dev)
    s_a = torch.empty(ma, dtype=torch.int64, device=dev)
    s_b = torch.empty(mb, dtype=torch.int64, device=dev)
    g = torch.empty((ma, mb), dtype=torch.float64, device=dev)
    g32 = torch.empty((mb, ma), dtype=torch.float32, device=dev) if want_f32 else None
    cpi.cpi_correlate(a, b, n, s_ab, s_a, s_b, g, g32, ws, stream)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    out = {"s_ab": s_ab.cpu(), "s_a": s_a.cpu(), "s_b": s_b.cpu(), "gamma": g.cpu()}
    if want_f32:
        out["gamma_f32"] = g32
    return out


def oracle_correlate(frames_host, la, lb, n, rows=None):
    import oracle

    return oracle.correlate(frames_host, la, frames_host, lb, n, rows=rows)


def make_frames(acq, device="cuda", n=None):
    A, B = synth.generate(acq, device, n_frames=n)
    fr, lay = synth.pack_side_by_side(A, B, acq.bits)
    return fr, lay


def assert_exact(got, want, rows=None):
    sl = slice(None) if rows is None else slice(rows[0], rows[1])
    assert np.array_equal(got["s_a"].numpy(), want["s_a"])
    assert np.array_equal(got["s_b"].numpy(), want["s_b"])
    gs = got["s_ab"].numpy()[sl]
    ws = want["s_ab"][sl]
    if not np.array_equal(gs, ws):
        bad = np.argwhere(gs != ws)
        i, j = bad[0]
        raise AssertionError(f"S_ab differs at {len(bad)} entries; first ({i},{j}): {gs[i, j]} != {ws[i, j]}")
    gg = got["gamma"].numpy()[sl]
    wg = want["gamma"][sl]
    # bit-identical doubles
    assert np.array_equal(gg.view(np.int64), wg.view(np.int64))


def refocus_gpu(g32, ha, wa, hb, wb, alpha, beta, stream=None):
    P = len(alpha)
    dev = g32.device
    ws = torch.empty(cpi.cpi_refocus_workspace_size(ha, wa, hb, wb, P), dtype=torch.uint8, device=dev)
    out = torch.empty((P, ha, wa), dtype=torch.float32, device=dev)
    cpi.cpi_refocus(g32, ha, wa, hb, wb, cpi.plane_array(alpha, beta), out, ws, stream)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    return out.cpu().double().numpy()


def refocus_tolerance(gamma64, ha, wa, hb, wb, alpha, beta):
    """Per-output bound 1e-6 * max|Gamma| * W_p(x), W_p(x) = total interpolation
    weight that falls inside the grid (the refocus of an all-ones Gamma)."""
    import oracle

    ones = np.ones((ha * wa, hb * wb))
    W = oracle.refocus(ones, ha, wa, hb, wb, alpha, beta)
    return 1e-6 * np.abs(gamma64).max() * W


def refocus_errors(out, ref, gamma64, ha, wa, hb, wb, alpha, beta):
    """Errors of a refocused stack against the FP64 oracle, in both readings of the
    refocusing target: the literal ratio max|R - R_fp64| / max|Gamma| and the
    per-unit-weight ratio max(|R - R_fp64| / (max|Gamma| W_p(x))) (<= 1 passes).
    Returns (literal, per_weight, tolerance array)."""
    tol = refocus_tolerance(gamma64, ha, wa, hb, wb, alpha, beta)
    err = np.abs(np.asarray(out, dtype=np.float64) - ref)
    gmax = np.abs(gamma64).max()
    literal = float(err.max() / gmax) if gmax > 0 else 0.0
    per_w = float((err / np.maximum(tol, 1e-300)).max())
    return literal, per_w, tol
