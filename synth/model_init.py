"""Seeded initial weights of the Gamma denoiser (an input of training, shared by
the tests, the benchmark and the smoke check; no part of the method's
arithmetic).

Model blob (float32, the library's layout): for each layer l = 0..3 the weights
W_l [Cout][Cin][3][3] then the biases b_l [Cout]; layers 9 -> 32 -> 32 -> 32 -> 1.
"""

from __future__ import annotations

import numpy as np

DENOISER_LAYERS = [(9, 32), (32, 32), (32, 32), (32, 1)]   # (Cin, Cout)
DENOISER_PARAMS = sum(co * ci * 9 + co for ci, co in DENOISER_LAYERS)   # 21409


def denoiser_init(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)) drawn from a Philox stream keyed by
    `seed`, zero biases, the last layer scaled by 0.1 so that the network starts
    close to the identity (its output is the centre channel plus a small
    correction)."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    parts = []
    for l, (ci, co) in enumerate(DENOISER_LAYERS):
        w = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (ci * 9))
        if l == len(DENOISER_LAYERS) - 1:
            w *= 0.1
        parts += [w.reshape(-1), np.zeros(co)]
    blob = np.concatenate(parts).astype(np.float32)
    assert blob.size == DENOISER_PARAMS
    return blob
