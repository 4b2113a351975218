"""Oracle of the Gamma denoiser (TEST INFRASTRUCTURE: only tests/, the smoke
check and bench.py's CPU baseline may import this module).

The paper has no denoiser; the network is the one the project specifies for
its "learned denoiser" row: it maps Gamma of Eq. (1) measured from few frames
to Gamma of many frames.  Plain numpy in float64, written for a reader to
check by eye:

* input of angular slice b = (br, bc): 9 channels, the Gamma slices of the 3 x 3
  angular neighbourhood (br + dy, bc + dx), dy, dx in {-1, 0, 1}, channel
  3 * (dy + 1) + (dx + 1), zero outside the angular grid, each a spatial image
  [ha][wa]; the whole Gamma is scaled by s = 1 / rms(Gamma_in) first;
* conv3x3(9 -> 32) + ReLU, conv3x3(32 -> 32) + ReLU, conv3x3(32 -> 32) + ReLU,
  conv3x3(32 -> 1), zero padding 1 (output the size of the input);
* output = centre channel (4) + last convolution; Gamma_out = output / s;
* training loss: mean over all outputs of (output - s * Gamma_target)^2.

BF16 points (where the kernels store bfloat16): the stacked input, every
weight (rounded from the float32 master copy when used), and every hidden
activation after its ReLU.  `bf16` rounds float64 -> float32 -> bfloat16
(round to nearest even at each step), as the kernels do from float32 values.
Biases stay float32; the output and every gradient stay unrounded.

Model blob (float32, the library's layout): for each layer l = 0..3 the weights
W_l [Cout][Cin][3][3] then the biases b_l [Cout].
"""

from __future__ import annotations

import numpy as np

LAYERS = [(9, 32), (32, 32), (32, 32), (32, 1)]   # (Cin, Cout)
N_PARAMS = sum(co * ci * 9 + co for ci, co in LAYERS)   # 21409


def bf16(x):
    """Round to bfloat16 (nearest even), via float32; returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def unpack(blob):
    """Model blob -> list of (W [Cout][Cin][3][3], b [Cout]) in float64."""
    blob = np.asarray(blob, dtype=np.float64)
    out, o = [], 0
    for ci, co in LAYERS:
        w = blob[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = blob[o:o + co]
        o += co
        out.append((w, b))
    assert o == N_PARAMS
    return out


def pack(params):
    return np.concatenate([np.concatenate([w.reshape(-1), b]) for w, b in params])


def scale_of(gamma):
    """s = 1 / rms(Gamma), in float64, then float32 (the kernels use a float32 s)."""
    g = np.asarray(gamma, dtype=np.float64)
    return float(np.float32(1.0 / np.sqrt(np.mean(g * g))))


def stack(gamma_slices, hb, wb, s):
    """gamma_slices [hb*wb][ha][wa] -> network input [hb*wb][9][ha][wa] (bf16)."""
    g = np.asarray(gamma_slices, dtype=np.float64)
    nb, ha, wa = g.shape
    assert nb == hb * wb
    x = np.zeros((nb, 9, ha, wa))
    for br in range(hb):
        for bc in range(wb):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    r, c = br + dy, bc + dx
                    if 0 <= r < hb and 0 <= c < wb:
                        x[br * wb + bc, 3 * (dy + 1) + (dx + 1)] = g[r * wb + c]
    return bf16(x * np.float32(s))


def conv3x3(x, w, b):
    """out[n, o, y, x] = b[o] + sum_{c, ky, kx} w[o, c, ky, kx] x[n, c, y + ky - 1, x + kx - 1]
    (zero padding)."""
    n, ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((n, w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + W])
    return out + b[None, :, None, None]


def forward(blob, x, exact=False):
    """Network on input x [n][9][H][W] (already bf16).  Returns (y [n][H][W],
    cache of the bf16 activations for the backward pass).  exact=True skips the
    bf16 roundings (a smooth function, for finite-difference checks)."""
    rnd = (lambda v: v) if exact else bf16
    params = [(rnd(w), b.astype(np.float64)) for w, b in unpack(blob)]
    acts = [x]
    a = x
    for w, b in params[:-1]:
        a = rnd(np.maximum(conv3x3(a, w, b), 0.0))
        acts.append(a)
    w, b = params[-1]
    y = x[:, 4] + conv3x3(a, w, b)[:, 0]
    return y, (params, acts)


def mse(y, t):
    """Loss and its gradient with respect to y."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(cache, dy):
    """Gradient of the loss with respect to the model blob (float64, blob layout)."""
    params, acts = cache
    grads = [None] * len(params)
    d = dy[:, None]                       # gradient at the last convolution's output
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        a = acts[l]                       # input of layer l
        n, ci, H, W = a.shape
        ap = np.pad(a, ((0, 0), (0, 0), (1, 1), (1, 1)))
        gw = np.zeros_like(w)
        for ky in range(3):
            for kx in range(3):
                gw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", d, ap[:, :, ky:ky + H, kx:kx + W])
        grads[l] = (gw, d.sum(axis=(0, 2, 3)))
        if l == 0:
            break
        # gradient at layer l's input: full correlation with the flipped kernel
        dp = np.pad(d, ((0, 0), (0, 0), (1, 1), (1, 1)))
        da = np.zeros_like(a)
        for ky in range(3):
            for kx in range(3):
                da += np.einsum("oc,nohw->nchw", w[:, :, ky, kx],
                                dp[:, :, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W])
        d = da * (a > 0)                  # through the ReLU that produced a
    return pack(grads)


def adam(blob, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), float64.  Returns (blob, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return blob - lr * mh / (np.sqrt(vh) + eps), m, v


def denoise(blob, gamma_slices, hb, wb):
    """Inference: Gamma slices [hb*wb][ha][wa] -> denoised slices, float64."""
    s = scale_of(gamma_slices)
    y, _ = forward(blob, stack(gamma_slices, hb, wb, s))
    return y / np.float32(s)


def loss_and_grad(blob, gamma_in, gamma_target, hb, wb):
    """Training loss of one Gamma and the gradient of the model blob."""
    s = scale_of(gamma_in)
    y, cache = forward(blob, stack(gamma_in, hb, wb, s))
    t = np.asarray(gamma_target, dtype=np.float64) * np.float32(s)
    loss, dy = mse(y, t)
    return loss, backward(cache, dy)
