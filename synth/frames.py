"""Chaotic-light frame generator and SwissSPAD2-style frame layout.

Source model (the paper gives none; this reading is recorded here and in the
design notes).  Per frame, a circular complex Gaussian field E ~ CN(0, I) is
drawn on an S x S source grid.

* Spatial detector A: |h * (M . E)|^2, where M is a fixed binary bar mask (the
  object) and h a normalised Gaussian blur (sigma 1.5 px, radius 5, zero
  padding), binned onto side_a x side_a detector pixels by summing the source
  pixels each detector pixel covers.
* Angular detector B: |fftshift(DFT2(E))|^2 (unnormalised DFT), binned the same
  way onto side_b x side_b pixels.
* Both intensities are scaled so that the pixel-averaged expected photon number
  per frame is ``mean_photons``; the scale uses the analytic expectation.
* Photon statistics: ``poisson8`` = Poisson counts clipped to 255 (uint8);
  ``bernoulli`` = 1-bit SPAD frames, P(click) = 1 - exp(-lambda);
  ``binomial255`` = sum of 255 binary sub-frames sharing the frame's lambda,
  i.e. Binomial(255, 1 - exp(-lambda)).

Frames are laid out as in Section 2 of the paper: each frame holds the two
images side by side (A on the left, B on the right), one byte per pixel for
counts or one bit per pixel, packed least-significant-bit first, for binary
frames.  Random numbers come from ``torch.Generator`` seeded per acquisition,
so a (seed, device type) pair always gives the same frames.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, replace
from typing import Optional

import numpy as np
import torch

_BATCH = 256  # frames simulated per batch; fixed so results do not depend on memory


@dataclass(frozen=True)
class Acquisition:
    side_a: int            # spatial detector is side_a x side_a pixels
    side_b: int            # angular detector is side_b x side_b pixels
    n_frames: int
    mean_photons: float    # pixel-averaged expected photons per pixel per frame
    counts: str            # 'poisson8' | 'bernoulli' | 'binomial255'
    src_side: Optional[int] = None   # default: 2 * max(side_a, side_b)
    sigma: float = 1.5
    radius: int = 5
    seed: int = 0
    mask_seed: Optional[int] = None  # None: the fixed three-bar object; else a seeded bar pattern

    @property
    def S(self) -> int:
        return self.src_side if self.src_side else 2 * max(self.side_a, self.side_b)

    @property
    def bits(self) -> int:
        return 1 if self.counts == "bernoulli" else 8


# The acquisition shapes of the benchmark workloads.
CONFIGS = {
    # 16x16 vs 16x16 uint8 Poisson counts, mean 2 photons, 2000 frames, 32x32 source
    "small_u8": Acquisition(16, 16, 2000, 2.0, "poisson8"),
    # 64x64 vs 32x32 binary SPAD frames, mean lambda 0.3, 20000 frames
    "spad_1bit": Acquisition(64, 32, 20000, 0.3, "bernoulli"),
    # 128x128 vs 64x64 uint8 sums of 255 binary sub-frames, 50000 frames
    "large_u8": Acquisition(128, 64, 50000, 0.3, "binomial255"),
}


def batched_acquisitions(n: int = 64, seed: int = 1234):
    """Uneven batch: side_a ~ U{32..96}, side_b ~ U{16..48}, N ~ U{5000..40000},
    uint8 Poisson counts with mean photons ~ U[1, 4]."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for i in range(n):
        sa = int(rng.integers(32, 97))
        sb = int(rng.integers(16, 49))
        nf = int(rng.integers(5000, 40001))
        mu = float(rng.uniform(1.0, 4.0))
        out.append(Acquisition(sa, sb, nf, mu, "poisson8", seed=seed * 1000 + i))
    return out


def uniform_planes(n_planes: int):
    """Uniformly spaced refocusing planes: alpha in [0.5, 1.5], beta = 1 - alpha.
    (alpha, beta) = (1, 0) is the plane the spatial detector is focused on."""
    if n_planes == 1:
        alpha = np.array([1.0])
    else:
        alpha = np.linspace(0.5, 1.5, n_planes)
    return alpha, 1.0 - alpha


# ----------------------------------------------------------------------------- model

def _bar_mask(S: int) -> np.ndarray:
    """Three vertical transmissive bars of width S/8, period S/4, centred."""
    m = np.zeros((S, S), dtype=np.float64)
    width = max(1, S // 8)
    period = max(2, S // 4)
    for k in (-1, 0, 1):
        c = S // 2 + k * period
        lo, hi = c - width // 2, c - width // 2 + width
        m[:, max(lo, 0):max(min(hi, S), 0)] = 1.0
    return m


def _random_bar_mask(S: int, mask_seed: int) -> np.ndarray:
    """2 to 4 transmissive bars, each vertical or horizontal, width S/16 .. S/6,
    at seeded positions (the union of them)."""
    rng = np.random.Generator(np.random.Philox(int(mask_seed)))
    m = np.zeros((S, S), dtype=np.float64)
    for _ in range(int(rng.integers(2, 5))):
        width = int(rng.integers(max(1, S // 16), max(2, S // 6) + 1))
        lo = int(rng.integers(0, S - width + 1))
        if rng.random() < 0.5:
            m[:, lo:lo + width] = 1.0
        else:
            m[lo:lo + width, :] = 1.0
    return m


def _mask(acq: "Acquisition") -> np.ndarray:
    return _bar_mask(acq.S) if acq.mask_seed is None else _random_bar_mask(acq.S, acq.mask_seed)


def _gauss1d(sigma: float, radius: int) -> np.ndarray:
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-0.5 * (x / sigma) ** 2)
    return g / g.sum()


def _bin_matrix(side: int, S: int) -> np.ndarray:
    """P[x, u] = 1 if source row/column u falls in detector row/column x."""
    u = np.arange(S)
    idx = (u * side) // S
    P = np.zeros((side, S), dtype=np.float64)
    P[idx, u] = 1.0
    return P


def _scales(acq: Acquisition):
    """Photon-number scale factors s_a, s_b from the analytic mean intensities."""
    S = acq.S
    g = _gauss1d(acq.sigma, acq.radius)
    M = _mask(acq)
    # E|F_a(u)|^2 = sum_v h(u - v)^2 M(v): zero-padded correlation of M with h^2
    g2 = g ** 2
    mean_grid = _conv_same_np(M, g2)
    Pa = _bin_matrix(acq.side_a, S)
    Ia = Pa @ mean_grid @ Pa.T
    s_a = acq.mean_photons / Ia.mean()
    Pb = _bin_matrix(acq.side_b, S)
    Ib = Pb @ np.full((S, S), float(S * S)) @ Pb.T
    s_b = acq.mean_photons / Ib.mean()
    return s_a, s_b


def _conv_same_np(img: np.ndarray, k1: np.ndarray) -> np.ndarray:
    """Separable zero-padded 'same' filtering with a symmetric 1-D kernel."""
    r = (len(k1) - 1) // 2
    S0, S1 = img.shape
    pad = np.zeros((S0 + 2 * r, S1 + 2 * r))
    pad[r:r + S0, r:r + S1] = img
    tmp = np.zeros((S0 + 2 * r, S1))
    for j, w in enumerate(k1):
        tmp += w * pad[:, j:j + S1]
    out = np.zeros((S0, S1))
    for j, w in enumerate(k1):
        out += w * tmp[j:j + S0, :]
    return out


def model_maps(acq: Acquisition):
    """Dense linear maps of the source model, for closed-form checks on small grids.

    Returns (L_a, L_b, Pa, Pb, s_a, s_b): L_a, L_b are [S*S, S*S] complex maps from
    the flattened source field to the flattened spatial / angular fields (row-major
    grid order, fftshifted frequencies for L_b); Pa, Pb are the 1-D binning
    matrices; s_a, s_b the photon scale factors."""
    S = acq.S
    if S > 48:
        raise ValueError("model_maps is meant for small source grids")
    g = _gauss1d(acq.sigma, acq.radius)
    r = acq.radius
    M = _mask(acq).reshape(-1)
    yy, xx = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    uy, ux = yy.reshape(-1), xx.reshape(-1)
    dy = uy[:, None] - uy[None, :]
    dx = ux[:, None] - ux[None, :]
    inside = (np.abs(dy) <= r) & (np.abs(dx) <= r)
    h = np.where(inside, g[np.clip(dy + r, 0, 2 * r)] * g[np.clip(dx + r, 0, 2 * r)], 0.0)
    L_a = (h * M[None, :]).astype(np.complex128)
    f = np.arange(S) - S // 2
    fy, fx = f[yy.reshape(-1)], f[xx.reshape(-1)]
    phase = -2j * np.pi * (fy[:, None] * uy[None, :] + fx[:, None] * ux[None, :]) / S
    L_b = np.exp(phase)
    s_a, s_b = _scales(acq)
    return L_a, L_b, _bin_matrix(acq.side_a, S), _bin_matrix(acq.side_b, S), s_a, s_b


def expected_gamma_counts(acq: Acquisition, device="cpu", n_frames: Optional[int] = None) -> torch.Tensor:
    """Expected value of Eq. (1) for Poisson counts, E[Gamma] = (1 - 1/N) Cov(A_a, B_b),
    as a float64 [side_a^2, side_b^2] tensor (the clip at 255 is ignored).

    For circular complex Gaussian E, Cov(|Psi_a(u)|^2, |Psi_b(v)|^2) = |K(u, v)|^2
    with K(u, v) = E[Psi_a(u) conj(Psi_b(v))] = (h * (M . exp(+2 pi i f_v . w / S)))(u):
    the blurred object modulated by the conjugate DFT basis vector of frequency v.
    Poisson noise adds no covariance between the two detectors.  Computed per band
    of frequency rows with the same separable blur as the generator, then binned."""
    if acq.counts != "poisson8":
        raise ValueError("closed form implemented for Poisson counts")
    device = torch.device(device)
    n = acq.n_frames if n_frames is None else n_frames
    S = acq.S
    s_a, s_b = _scales(acq)
    g = torch.tensor(_gauss1d(acq.sigma, acq.radius), dtype=torch.float32, device=device)
    M = torch.tensor(_mask(acq), dtype=torch.float32, device=device)
    Pa = torch.tensor(_bin_matrix(acq.side_a, S), dtype=torch.float64, device=device)
    Pb = torch.tensor(_bin_matrix(acq.side_b, S), dtype=torch.float64, device=device)
    w = torch.arange(S, dtype=torch.float64, device=device)
    f = torch.arange(S, dtype=torch.float64, device=device) - S // 2
    cov = torch.zeros((acq.side_a * acq.side_a, acq.side_b * acq.side_b), dtype=torch.float64, device=device)
    ey = torch.exp(2j * math.pi * f[:, None] * w[None, :] / S)          # [fy, wy]
    ex = ey                                                              # [fx, wx]
    for fy0 in range(0, S, 8):
        fys = slice(fy0, min(fy0 + 8, S))
        ny = fys.stop - fys.start
        # modulated object for every (fy, fx) of the band: [ny, S(fx), S(wy), S(wx)]
        mod = (ey[fys][:, None, :, None] * ex[None, :, None, :]).to(torch.complex64) * M
        K = _blur_complex(mod.reshape(ny * S, S, S), g, acq.radius)
        P2 = (K.real.double() ** 2 + K.imag.double() ** 2).reshape(ny, S, S, S)   # [fy, fx, uy, ux]
        Ia = torch.einsum("au,yxuv,bv->yxab", Pa, P2, Pa).reshape(ny, S, -1)    # [fy, fx, a]
        by = (torch.arange(fys.start, fys.stop, device=device) * acq.side_b) // S
        Ib = torch.einsum("yxa,cx->yac", Ia, Pb)                                 # [fy, a, bx]
        for k in range(ny):
            cov[:, int(by[k]) * acq.side_b:(int(by[k]) + 1) * acq.side_b] += Ib[k]
    return cov * (s_a * s_b) * (1.0 - 1.0 / n)


# ----------------------------------------------------------------------------- sampling

def _blur_complex(field: torch.Tensor, g: torch.Tensor, r: int) -> torch.Tensor:
    """Zero-padded separable Gaussian filtering of a complex [n, S, S] field."""
    n, S, _ = field.shape
    x = torch.view_as_real(field).permute(0, 3, 1, 2).reshape(n * 2, 1, S, S)
    x = torch.nn.functional.conv2d(x, g.view(1, 1, -1, 1), padding=(r, 0))
    x = torch.nn.functional.conv2d(x, g.view(1, 1, 1, -1), padding=(0, r))
    x = x.reshape(n, 2, S, S).permute(0, 2, 3, 1).contiguous()
    return torch.view_as_complex(x)


def generate(acq: Acquisition, device="cpu", n_frames: Optional[int] = None):
    """Simulate the acquisition. Returns (A, B): uint8 tensors [n, side_a, side_a]
    and [n, side_b, side_b] on ``device`` (0/1 values for binary frames)."""
    device = torch.device(device)
    n_total = acq.n_frames if n_frames is None else n_frames
    S = acq.S
    s_a, s_b = _scales(acq)
    dt = torch.float32
    g = torch.tensor(_gauss1d(acq.sigma, acq.radius), dtype=dt, device=device)
    M = torch.tensor(_mask(acq), dtype=dt, device=device)
    Pa = torch.tensor(_bin_matrix(acq.side_a, S), dtype=dt, device=device)
    Pb = torch.tensor(_bin_matrix(acq.side_b, S), dtype=dt, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(acq.seed))
    A = torch.empty((n_total, acq.side_a, acq.side_a), dtype=torch.uint8, device=device)
    B = torch.empty((n_total, acq.side_b, acq.side_b), dtype=torch.uint8, device=device)
    for f0 in range(0, n_total, _BATCH):
        nb = min(_BATCH, n_total - f0)
        re = torch.randn((nb, S, S), generator=gen, dtype=dt, device=device)
        im = torch.randn((nb, S, S), generator=gen, dtype=dt, device=device)
        E = torch.complex(re, im) * (1.0 / math.sqrt(2.0))
        Fa = _blur_complex(E * M, g, acq.radius)
        Fb = torch.fft.fftshift(torch.fft.fft2(E), dim=(-2, -1))
        Ia = Pa @ (Fa.real ** 2 + Fa.imag ** 2) @ Pa.T
        Ib = Pb @ (Fb.real ** 2 + Fb.imag ** 2) @ Pb.T
        A[f0:f0 + nb] = _photons(Ia * s_a, acq.counts, gen)
        B[f0:f0 + nb] = _photons(Ib * s_b, acq.counts, gen)
    return A, B


def _photons(lam: torch.Tensor, kind: str, gen: torch.Generator) -> torch.Tensor:
    lam = lam.clamp_min(0.0)
    if kind == "poisson8":
        return torch.poisson(lam, generator=gen).clamp_(max=255).to(torch.uint8)
    p = -torch.expm1(-lam)
    if kind == "bernoulli":
        return torch.bernoulli(p, generator=gen).to(torch.uint8)
    if kind == "binomial255":
        cnt = torch.full_like(p, 255.0)
        return torch.binomial(cnt, p, generator=gen).to(torch.uint8)
    raise ValueError(kind)


# ----------------------------------------------------------------------------- layout

def pack_bits_lsb(x: torch.Tensor) -> torch.Tensor:
    """Pack 0/1 values along the last axis into bytes, least significant bit first.
    The last axis must be a multiple of 8."""
    *lead, n = x.shape
    assert n % 8 == 0
    w = torch.tensor([1, 2, 4, 8, 16, 32, 64, 128], dtype=torch.int32, device=x.device)
    y = (x.reshape(*lead, n // 8, 8).to(torch.int32) * w).sum(-1)
    return y.to(torch.uint8)


def pack_side_by_side(A: torch.Tensor, B: torch.Tensor, bits: int):
    """Lay each frame out as one H x (W_a + W_b) image, A on the left and B on the
    right (Section 2 of the paper), rows of H = max(H_a, H_b); unused pixels are 0.

    Returns (frames, layout): frames is a uint8 tensor [n, frame_bytes]; layout
    gives, per image, the ROI origin (x0, y0), size, the row stride in pixels and
    the frame stride in bytes, i.e. the fields of the library's frame descriptor."""
    n, ha, wa = A.shape
    _, hb, wb = B.shape
    H, W = max(ha, hb), wa + wb
    img = torch.zeros((n, H, W), dtype=torch.uint8, device=A.device)
    img[:, :ha, :wa] = A
    img[:, :hb, wa:] = B
    if bits == 8:
        frames = img.reshape(n, H * W)
        frame_bytes = H * W
    elif bits == 1:
        nbits = H * W
        pad = (-nbits) % 8
        flat = img.reshape(n, nbits)
        if pad:
            flat = torch.cat([flat, flat.new_zeros((n, pad))], dim=1)
        frames = pack_bits_lsb(flat)
        frame_bytes = (nbits + pad) // 8
    else:
        raise ValueError(bits)
    common = dict(bits=bits, row_stride=W, frame_stride_bytes=frame_bytes, bit_order=0)
    layout = {
        "a": dict(height=ha, width=wa, x0=0, y0=0, **common),
        "b": dict(height=hb, width=wb, x0=wa, y0=0, **common),
        "frame_bytes": frame_bytes,
    }
    return frames.contiguous(), layout


def bin_file_frames(n: int, seed: int, height: int = 256, width: int = 512, p: float = 0.1, device="cpu"):
    """Binary frames in the layout of the paper's .bin files (Section 2): each frame
    is height x width pixels, two side-by-side images (A: columns 0 .. width/2 - 1,
    B: the rest), 1 bit per pixel, rows packed least-significant-bit first.

    For scale runs, where the source model would cost a 2-D FFT of the whole
    source grid per frame: pixels are Bernoulli(p_i) with a per-frame intensity
    p_i = p (1 + 0.5 u_i), u_i uniform on [-1, 1], shared by both images, so
    every pixel pair is positively correlated (Gamma = Var(p_i) > 0).  Returns a
    uint8 tensor [n, height * width / 8]."""
    device = torch.device(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty((n, height * width // 8), dtype=torch.uint8, device=device)
    for f0 in range(0, n, _BATCH):
        nb = min(_BATCH, n - f0)
        pi = p * (1.0 + 0.5 * (2.0 * torch.rand((nb, 1), generator=gen, device=device) - 1.0))
        bits = (torch.rand((nb, height * width), generator=gen, device=device) < pi).to(torch.uint8)
        out[f0:f0 + nb] = pack_bits_lsb(bits)
    return out


def bin_file_layout(height: int = 256, width: int = 512):
    """Frame descriptors of the two images of bin_file_frames (fields of cpi_frames)."""
    half = width // 2
    common = dict(bits=1, height=height, width=half, y0=0, row_stride=width,
                  frame_stride_bytes=height * width // 8, bit_order=0)
    return {"a": dict(x0=0, **common), "b": dict(x0=half, **common)}


def with_seed(acq: Acquisition, seed: int) -> Acquisition:
    return replace(acq, seed=seed)


def random_gamma(ma: int, mb: int, seed: int) -> np.ndarray:
    """A seeded stand-in correlation function for refocusing checks: float64
    [ma][mb] (row = spatial pixel, column = angular pixel), i.i.d. standard
    normal values rounded to float32 (so that the FP32 copy a GPU path reads is
    the same data).  Refocusing cost does not depend on the values."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    return rng.standard_normal((ma, mb), dtype=np.float32).astype(np.float64)
