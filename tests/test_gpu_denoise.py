"""GPU parity of the Gamma denoiser against its oracle (oracle/denoiser.py).

Both sides round the stacked input, the weights in use and the hidden
activations to bfloat16 at the same points; the remaining differences are the
order of float32 sums (FP32 on the GPU, float64 in the oracle) and the rare
bfloat16 rounding that this order moves across a rounding boundary (one
activation then differs by one bfloat16 unit, 2^-8 of its size, which reaches
an output through weights of order 0.1).  Tolerances: outputs within 2e-3 of
the largest output (mean difference below 2e-5 of it); gradients, layer by
layer, within 2e-3 of the layer's largest gradient component."""

import numpy as np
import pytest
import torch

import paper_2407_20692_gb300 as cpi
import synth
from oracle import denoiser as dn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready):
    yield


def _model(seed, noise=0.05):
    rng = np.random.default_rng(seed)
    blob = synth.denoiser_init(seed).astype(np.float64) + noise * rng.standard_normal(dn.N_PARAMS)
    return blob.astype(np.float32)


def _gamma(seed, hb, wb, ha, wa):
    """Smooth-ish random Gamma slices plus noise, float32 [hb*wb][ha*wa]."""
    rng = np.random.default_rng(seed)
    base = rng.standard_normal((hb * wb, ha, wa))
    base = base + np.roll(base, 1, axis=1) + np.roll(base, 1, axis=2)
    return (0.01 * base).astype(np.float32).reshape(hb * wb, ha * wa)


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def test_denoise_forward_matches_oracle_small():
    hb, wb, ha, wa = 3, 4, 12, 20
    blob = _model(1)
    g = _gamma(2, hb, wb, ha, wa)
    ws = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(_dev(g))
    cpi.cpi_denoise(_dev(blob), _dev(g), out, ha, wa, hb, wb, ws)
    torch.cuda.synchronize()
    want = dn.denoise(blob, g.reshape(-1, ha, wa), hb, wb).reshape(hb * wb, -1)
    s = dn.scale_of(g)
    d = np.abs(out.cpu().numpy() - want) * s                 # in units of the network output y
    ymax = np.abs(want).max() * s
    assert d.max() <= 2e-3 * ymax, d.max() / ymax
    assert d.mean() <= 2e-5 * ymax, d.mean() / ymax


def test_denoise_forward_matches_oracle_on_sampled_slices_of_the_full_workload():
    """64x64 spatial vs 32x32 angular: the oracle evaluates the network on a few
    slices (corners, edges, interior), the GPU on all 1024."""
    hb = wb = 32
    ha = wa = 64
    blob = _model(3)
    g = _gamma(4, hb, wb, ha, wa)
    ws = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(_dev(g))
    cpi.cpi_denoise(_dev(blob), _dev(g), out, ha, wa, hb, wb, ws)
    torch.cuda.synchronize()
    s = dn.scale_of(g)
    x = dn.stack(g.reshape(-1, ha, wa), hb, wb, s)
    idx = np.array([0, wb - 1, (hb - 1) * wb, hb * wb - 1, 5, 17 * wb, 17 * wb + wb - 1, 500, 777])
    y, _ = dn.forward(blob, x[idx])
    got = out.cpu().numpy()[idx].reshape(len(idx), ha, wa) * s
    d = np.abs(got - y)
    ymax = np.abs(y).max()
    assert d.max() <= 2e-3 * ymax, d.max() / ymax
    assert d.mean() <= 2e-5 * ymax, d.mean() / ymax


@pytest.mark.parametrize("hb,wb,ha,wa", [(2, 3, 10, 32), (2, 2, 5, 128)])
def test_denoise_forward_tensor_core_widths_match_oracle(hb, wb, ha, wa):
    """Widths 32 and 128 (the tensor-core layers; 64 is the workload test), with
    row counts that leave the last row block of a slice ragged."""
    blob = _model(12)
    g = _gamma(13 + wa, hb, wb, ha, wa)
    ws = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(_dev(g))
    cpi.cpi_denoise(_dev(blob), _dev(g), out, ha, wa, hb, wb, ws)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    want = dn.denoise(blob, g.reshape(-1, ha, wa), hb, wb).reshape(hb * wb, -1)
    s = dn.scale_of(g)
    d = np.abs(out.cpu().numpy() - want) * s
    ymax = np.abs(want).max() * s
    assert d.max() <= 2e-3 * ymax, d.max() / ymax
    assert d.mean() <= 2e-5 * ymax, d.mean() / ymax


def test_denoise_gradient_through_tensor_core_forward_matches_oracle():
    hb, wb, ha, wa = 2, 2, 8, 32
    blob = _model(14)
    g = _gamma(15, hb, wb, ha, wa)
    t = _gamma(16, hb, wb, ha, wa) * 0.5 + g * 0.5
    got, loss = _grad(blob, g, t, hb, wb, ha, wa)
    want_loss, want = dn.loss_and_grad(blob, g.reshape(-1, ha, wa), t.reshape(-1, ha, wa), hb, wb)
    assert abs(loss - want_loss) <= 1e-4 * want_loss
    o = 0
    for ci, co in dn.LAYERS:
        n = co * ci * 9 + co
        gl, wl = got[o:o + n], want[o:o + n]
        assert np.abs(gl - wl).max() <= 2e-3 * np.abs(wl).max(), (ci, co, np.abs(gl - wl).max() / np.abs(wl).max())
        o += n


def test_denoise_gradient_tensor_core_weight_gradients_match_oracle():
    """Images 64 pixels wide take the tensor-core weight gradients (delta split
    into two bf16 terms, x-shifted input copies, one GEMM over the pixels per
    layer); 40 rows make a ragged second block of rows.  Same tolerance as the
    float32 path, and bit-identical on a second run."""
    hb, wb, ha, wa = 2, 3, 40, 64
    blob = _model(21)
    g = _gamma(22, hb, wb, ha, wa)
    t = _gamma(23, hb, wb, ha, wa) * 0.5 + g * 0.5
    got, loss = _grad(blob, g, t, hb, wb, ha, wa)
    want_loss, want = dn.loss_and_grad(blob, g.reshape(-1, ha, wa), t.reshape(-1, ha, wa), hb, wb)
    assert abs(loss - want_loss) <= 1e-4 * want_loss
    o = 0
    for ci, co in dn.LAYERS:
        n = co * ci * 9 + co
        gl, wl = got[o:o + n], want[o:o + n]
        assert np.abs(gl - wl).max() <= 2e-3 * np.abs(wl).max(), (ci, co, np.abs(gl - wl).max() / np.abs(wl).max())
        o += n
    again, loss2 = _grad(blob, g, t, hb, wb, ha, wa)
    assert np.array_equal(got.view(np.uint32), again.view(np.uint32)) and loss2 == loss


def test_denoise_tensor_core_weight_gradients_over_many_units():
    """192 slices of 16 x 64: more row units than CTAs, so CTAs accumulate several
    units in tensor memory before writing their partial sums."""
    hb, wb, ha, wa = 8, 24, 16, 64
    blob = _model(31)
    g = _gamma(32, hb, wb, ha, wa)
    t = _gamma(33, hb, wb, ha, wa) * 0.5 + g * 0.5
    got, loss = _grad(blob, g, t, hb, wb, ha, wa)
    want_loss, want = dn.loss_and_grad(blob, g.reshape(-1, ha, wa), t.reshape(-1, ha, wa), hb, wb)
    assert abs(loss - want_loss) <= 1e-4 * want_loss
    o = 0
    for ci, co in dn.LAYERS:
        n = co * ci * 9 + co
        gl, wl = got[o:o + n], want[o:o + n]
        assert np.abs(gl - wl).max() <= 2e-3 * np.abs(wl).max(), (ci, co, np.abs(gl - wl).max() / np.abs(wl).max())
        o += n


def _grad(blob, g, t, hb, wb, ha, wa):
    ws = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb, training=True), dtype=torch.uint8,
                     device="cuda")
    grad = torch.empty(cpi.DENOISER_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    cpi.cpi_denoise_grad(_dev(blob), _dev(g), _dev(t), ha, wa, hb, wb, grad, loss, ws)
    torch.cuda.synchronize()
    return grad.cpu().numpy(), float(loss.item())


def test_denoise_gradient_matches_oracle_and_is_deterministic():
    hb, wb, ha, wa = 3, 5, 16, 24
    blob = _model(5)
    g = _gamma(6, hb, wb, ha, wa)
    t = _gamma(7, hb, wb, ha, wa) * 0.5 + g * 0.5
    got, loss = _grad(blob, g, t, hb, wb, ha, wa)
    want_loss, want = dn.loss_and_grad(blob, g.reshape(-1, ha, wa), t.reshape(-1, ha, wa), hb, wb)
    assert abs(loss - want_loss) <= 1e-4 * want_loss
    o = 0
    for ci, co in dn.LAYERS:
        n = co * ci * 9 + co
        gl, wl = got[o:o + n], want[o:o + n]
        assert np.abs(gl - wl).max() <= 2e-3 * np.abs(wl).max(), (ci, co, np.abs(gl - wl).max() / np.abs(wl).max())
        o += n
    again, loss2 = _grad(blob, g, t, hb, wb, ha, wa)
    assert np.array_equal(got.view(np.uint32), again.view(np.uint32)) and loss2 == loss


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(8)
    n = cpi.DENOISER_PARAMS
    w = rng.standard_normal(n).astype(np.float32)
    m = (0.01 * rng.standard_normal(n)).astype(np.float32)
    v = (1e-4 * rng.random(n)).astype(np.float32)
    g = (0.1 * rng.standard_normal(n)).astype(np.float32)
    dw, dm, dv = _dev(w), _dev(m), _dev(v)
    cpi.cpi_denoise_adam(dw, dm, dv, _dev(g), 3, 1e-3)
    torch.cuda.synchronize()
    w2, m2, v2 = dn.adam(w.astype(np.float64), m.astype(np.float64), v.astype(np.float64), g.astype(np.float64),
                         3, 1e-3)
    # FP32 against float64: a few roundings of each term (0.9 m + 0.1 g can cancel,
    # so the bound is on the size of the terms, not of the result)
    u = 2.0 ** -24
    tm = 0.9 * np.abs(m) + 0.1 * np.abs(g)
    tv = 0.999 * np.abs(v) + 0.001 * g.astype(np.float64) ** 2
    assert (np.abs(dm.cpu().numpy() - m2) <= 8 * u * tm).all()
    assert (np.abs(dv.cpu().numpy() - v2) <= 8 * u * tv).all()
    step_size = np.abs(w2 - w)
    assert (np.abs(dw.cpu().numpy() - w2) <= 8 * u * (np.abs(w) + step_size) + 64 * u * step_size).all()


def test_training_steps_reduce_the_loss():
    hb, wb, ha, wa = 4, 4, 16, 16
    rng = np.random.default_rng(9)
    clean = _gamma(10, hb, wb, ha, wa)
    noisy = (clean + 0.01 * rng.standard_normal(clean.shape)).astype(np.float32)
    model = _dev(synth.denoiser_init(11))
    m = torch.zeros_like(model)
    v = torch.zeros_like(model)
    ws = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb, training=True), dtype=torch.uint8,
                     device="cuda")
    grad = torch.empty_like(model)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    gi, gt = _dev(noisy), _dev(clean)
    losses = []
    for step in range(1, 61):
        cpi.cpi_denoise_grad(model, gi, gt, ha, wa, hb, wb, grad, loss, ws)
        cpi.cpi_denoise_adam(model, m, v, grad, step, 3e-3)
        losses.append(float(loss.item()))
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def test_denoise_argument_errors():
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    x = torch.zeros(64, device="cuda")
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_denoise(x, x, x, 0, 8, 2, 2, ws)
    assert e.value.code == 1
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_denoise(x, x, x, 8, 8, 2, 2, ws)            # workspace too small
    assert e.value.code == 3
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_denoise_adam(x, x, x, x, 0, 1e-3)           # steps count from 1
    assert e.value.code == 1


def _gamma_prefixes(acq, prefixes):
    import synth

    A, B = synth.generate(acq, "cuda")
    fr, lay = synth.pack_side_by_side(A, B, 8)
    la, lb = lay["a"], lay["b"]
    mk = lambda l: cpi.frames(fr, 8, l["height"], l["width"], l["x0"], l["y0"], l["row_stride"],
                              l["frame_stride_bytes"])
    a, b = mk(la), mk(lb)
    ma, mb = la["height"] * la["width"], lb["height"] * lb["width"]
    s_ab = torch.empty((ma, mb), dtype=torch.int64, device="cuda")
    s_a = torch.empty(ma, dtype=torch.int64, device="cuda")
    s_b = torch.empty(mb, dtype=torch.int64, device="cuda")
    g64 = torch.empty((ma, mb), dtype=torch.float64, device="cuda")
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, max(prefixes)), dtype=torch.uint8, device="cuda")
    out = []
    for k in prefixes:
        g32 = torch.empty((mb, ma), dtype=torch.float32, device="cuda")
        cpi.cpi_correlate(a, b, k, s_ab, s_a, s_b, g64, g32, ws)
        out.append(g32)
    return out


def test_committed_model_refocuses_better_from_5000_frames_than_plain_gamma_from_50000():
    """The trained model shipped with the library (trained on Gamma from 1000
    frames of seeded objects, targets the closed-form expected Gamma): on a seed
    outside its training set, the refocused stack of the denoised Gamma from 5000
    frames is closer to the refocused closed form than that of the plain Gamma
    from 50000 frames, and closer than zeros."""
    import os

    import synth

    path = os.path.join(os.path.dirname(cpi.__file__), "models", "denoiser_64x64_32x32_n1000.npy")
    model = _dev(np.load(path))
    ha = wa = 64
    hb = wb = 32
    acq = synth.Acquisition(64, 32, 50000, 2.0, "poisson8", seed=777001, mask_seed=777001)
    g5k, g50k = _gamma_prefixes(acq, [5000, 50000])
    ref = synth.expected_gamma_counts(acq, "cuda", n_frames=10 ** 12).t().contiguous().to(torch.float32)
    ws = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb), dtype=torch.uint8, device="cuda")
    den = torch.empty_like(g5k)
    cpi.cpi_denoise(model, g5k, den, ha, wa, hb, wb, ws)
    alpha, beta = synth.uniform_planes(32)
    planes = cpi.plane_array(alpha, beta)
    rws = torch.empty(cpi.cpi_refocus_workspace_size(ha, wa, hb, wb, 32), dtype=torch.uint8, device="cuda")

    def refocused(g):
        r = torch.empty((32, ha, wa), dtype=torch.float32, device="cuda")
        cpi.cpi_refocus(g, ha, wa, hb, wb, planes, r, rws)
        return r.double()

    r_ref = refocused(ref)
    err = lambda g: float(torch.linalg.vector_norm(refocused(g) - r_ref) / torch.linalg.vector_norm(r_ref))
    e_den, e_plain = err(den), err(g50k)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    assert e_den < e_plain and e_den < 1.0, (e_den, e_plain)
