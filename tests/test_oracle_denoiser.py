"""Pins of the denoiser oracle (CPU): bfloat16 rounding against torch's
conversion, the convolution against scipy's 2-D correlation, the angular
neighbourhood stacking by construction, the backward pass against central
finite differences of the unrounded network, Adam against its closed form,
and the closed-form expected Gamma used as training target and error reference
against the dense linear-map formula."""

import numpy as np
import pytest
import torch

import synth
from oracle import denoiser as dn


def test_bf16_matches_torch_round_to_nearest_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0, 65504.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(dn.bf16(x), want)
    assert dn.bf16(1.0 + 2.0 ** -8) == 1.0                  # tie -> even
    assert dn.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # tie -> even (up)


def test_conv3x3_is_scipy_correlation_summed_over_channels():
    from scipy.signal import correlate2d

    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 7, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = dn.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(correlate2d(x[n, c], w[o, c], mode="same", boundary="fill") for c in range(3))
            assert np.allclose(got[n, o], want, rtol=0, atol=1e-12)


def test_stack_takes_the_3x3_angular_neighbourhood_with_zero_fill():
    hb, wb, ha, wa = 3, 4, 2, 2
    g = np.stack([np.full((ha, wa), float(1 + b)) for b in range(hb * wb)])
    x = dn.stack(g, hb, wb, 1.0)
    for br in range(hb):
        for bc in range(wb):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    r, c = br + dy, bc + dx
                    want = 1 + r * wb + c if (0 <= r < hb and 0 <= c < wb) else 0.0
                    assert (x[br * wb + bc, 3 * (dy + 1) + (dx + 1)] == want).all()


def _tiny(seed):
    rng = np.random.default_rng(seed)
    hb, wb, ha, wa = 2, 3, 5, 4
    blob = synth.denoiser_init(seed).astype(np.float64)
    blob += 0.05 * rng.standard_normal(blob.size)      # non-zero biases, a non-trivial last layer
    x = rng.standard_normal((hb * wb, 9, ha, wa))
    t = rng.standard_normal((hb * wb, ha, wa))
    return blob, x, t


def test_backward_matches_finite_differences_of_the_unrounded_network():
    blob, x, t = _tiny(2)

    def loss(b):
        y, _ = dn.forward(b, x, exact=True)
        return dn.mse(y, t)[0]

    y, cache = dn.forward(blob, x, exact=True)
    _, dy = dn.mse(y, t)
    g = dn.backward(cache, dy)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(dn.N_PARAMS, 60, replace=False),
                          [dn.N_PARAMS - 1, 0, 2592, 2592 + 31]])   # last bias, first weight, layer-0 biases
    h = 1e-6
    for i in idx:
        e = np.zeros_like(blob)
        e[i] = h
        fd = (loss(blob + e) - loss(blob - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_last_layer_returns_the_centre_channel():
    blob, x, _ = _tiny(4)
    p = dn.unpack(blob)
    p[-1] = (np.zeros_like(p[-1][0]), np.zeros(1))
    y, _ = dn.forward(dn.pack(p), dn.bf16(x))
    assert np.array_equal(y, dn.bf16(x)[:, 4])


def test_adam_closed_form():
    w0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    w1, m1, v1 = dn.adam(w0, m, v, g, 1, lr, b1, b2, eps)
    # step 1: bias-corrected moments are g and g^2
    assert np.allclose(w1, w0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    w2, _, _ = dn.adam(w1, m1, v1, g, 2, lr, b1, b2, eps)
    # constant gradient: the corrected moments stay g and g^2
    assert np.allclose(w2, w1 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)


def test_expected_gamma_matches_the_dense_linear_map_formula():
    import synth

    acq = synth.Acquisition(8, 8, 1000, 2.0, "poisson8", mask_seed=5)
    La, Lb, Pa, Pb, s_a, s_b = synth.model_maps(acq)
    K2 = np.abs(La @ Lb.conj().T) ** 2                        # |E[Psi_a(u) conj(Psi_b(v))]|^2
    S = acq.S
    Ba = np.kron(Pa, Pa)                                      # source pixel -> detector pixel (row-major)
    Bb = np.kron(Pb, Pb)
    want = (1 - 1 / acq.n_frames) * s_a * s_b * (Ba @ K2 @ Bb.T)
    got = synth.expected_gamma_counts(acq).numpy()
    assert got.shape == want.shape == (64, 64)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-9 * np.abs(want).max())
