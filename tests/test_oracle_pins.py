"""Pins of the CPU oracle to facts outside itself (no GPU).

Eq. (1) is pinned by exact rational evaluation on hand-worked inputs, by
numpy's biased covariance (a library routine that computes Eq. (1) in floating
point), by exact invariants, and statistically by the closed-form correlation of
the chaotic-light source model (Gaussian moment theorem / Laplace transform of
Gaussian quadratic forms).  Refocusing is pinned by hand-worked values, by
scipy's linear spline interpolation with zero padding, and by special planes
that reduce to row sums and integer gathers.
"""

import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _desc(d, lay):
    return dict(bits=lay["bits"], row_stride=lay["row_stride"],
                frame_stride_bytes=lay["frame_stride_bytes"], bit_order=lay.get("bit_order", 0), **d)


def _eq1_exact(ua, ub):
    """Eq. (1) literally, in exact rationals: mean(A B) - mean(A) mean(B)."""
    n = ua.shape[1]
    out = []
    for a in range(ua.shape[0]):
        row = []
        for b in range(ub.shape[0]):
            mab = Fraction(int(np.dot(ua[a].astype(np.int64), ub[b].astype(np.int64))), n)
            ma = Fraction(int(ua[a].astype(np.int64).sum()), n)
            mb = Fraction(int(ub[b].astype(np.int64).sum()), n)
            row.append(mab - ma * mb)
        out.append(row)
    return out


def _frames(acq, n=None):
    A, B = synth.generate(acq, "cpu", n_frames=n)
    fr, lay = synth.pack_side_by_side(A, B, acq.bits)
    return A, B, fr.numpy(), lay


# ----------------------------------------------------------------------------- Eq. (1)

@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "eq1_hand.json")))["cases"],
                         ids=lambda c: c["name"])
def test_eq1_hand_worked(oracle_mod, case):
    fr = np.array(case["frames"], dtype=np.uint8)
    lay = dict(bits=case["bits"], row_stride=case["row_stride"],
               frame_stride_bytes=case["frame_stride_bytes"], bit_order=case["bit_order"])
    da, db = _desc(case["a"], lay), _desc(case["b"], lay)
    r = oracle_mod.correlate(fr, da, fr, db, len(fr))
    assert r["s_a"].tolist() == case["s_a"]
    assert r["s_b"].tolist() == case["s_b"]
    assert r["s_ab"].tolist() == case["s_ab"]
    want = np.array([[float(Fraction(x)) for x in row] for row in case["gamma"]])
    assert np.array_equal(r["gamma"], want)


@pytest.mark.parametrize("name,n", [("small_u8", 300), ("spad_1bit", 200)])
def test_eq1_exact_rationals(oracle_mod, name, n):
    """Brute force: every Gamma entry equals the correctly rounded exact value."""
    acq = synth.CONFIGS[name]
    acq = synth.frames.replace(acq, side_a=8 if name == "spad_1bit" else acq.side_a,
                               side_b=4 if name == "spad_1bit" else 6, src_side=24, seed=3)
    A, B, fr, lay = _frames(acq, n)
    r = oracle_mod.correlate(fr, lay["a"], fr, lay["b"], n)
    ua = A.reshape(n, -1).T.numpy()
    ub = B.reshape(n, -1).T.numpy()
    exact = _eq1_exact(ua, ub)
    want = np.array([[float(x) for x in row] for row in exact])
    assert np.array_equal(r["gamma"], want)
    assert np.array_equal(r["s_a"], ua.astype(np.int64).sum(1))
    assert np.array_equal(r["s_ab"], ua.astype(np.int64) @ ub.astype(np.int64).T)


def test_eq1_matches_numpy_biased_covariance(oracle_mod):
    acq = synth.frames.replace(synth.CONFIGS["small_u8"], side_a=8, side_b=8, src_side=16, seed=5)
    n = 1000
    A, B, fr, lay = _frames(acq, n)
    r = oracle_mod.correlate(fr, lay["a"], fr, lay["b"], n)
    X = np.concatenate([A.reshape(n, -1).numpy(), B.reshape(n, -1).numpy()], 1).astype(np.float64)
    C = np.cov(X.T, bias=True)
    ma = A[0].numel()
    cross = C[:ma, ma:]
    scale = np.abs(cross).max()
    assert np.max(np.abs(r["gamma"] - cross)) <= 1e-12 * max(scale, 1.0)


def test_eq1_invariants(oracle_mod):
    acq = synth.frames.replace(synth.CONFIGS["small_u8"], side_a=6, side_b=4, src_side=12, seed=11)
    n = 500
    A, B, fr, lay = _frames(acq, n)
    base = oracle_mod.correlate(fr, lay["a"], fr, lay["b"], n)
    # frame order does not matter (sums are exact)
    perm = np.random.default_rng(0).permutation(n)
    r = oracle_mod.correlate(fr[perm], lay["a"], fr[perm], lay["b"], n)
    assert np.array_equal(r["gamma"], base["gamma"])
    # swapping the detectors transposes Gamma
    r = oracle_mod.correlate(fr, lay["b"], fr, lay["a"], n)
    assert np.array_equal(r["gamma"], base["gamma"].T)
    # a constant offset on A leaves Gamma unchanged exactly
    A2 = (A.to(torch.int32) + 7).clamp(max=255).to(torch.uint8)
    assert int(A.max()) + 7 <= 255
    fr2, lay2 = synth.pack_side_by_side(A2, B, 8)
    r = oracle_mod.correlate(fr2.numpy(), lay2["a"], fr2.numpy(), lay2["b"], n)
    assert np.array_equal(r["gamma"], base["gamma"])
    # doubling A doubles Gamma exactly
    fr3, lay3 = synth.pack_side_by_side(A * 2, B, 8)
    r = oracle_mod.correlate(fr3.numpy(), lay3["a"], fr3.numpy(), lay3["b"], n)
    assert np.array_equal(r["gamma"], 2.0 * base["gamma"])
    # identical detectors: symmetric, positive semi-definite
    r = oracle_mod.correlate(fr, lay["a"], fr, lay["a"], n)
    g = r["gamma"]
    assert np.array_equal(g, g.T)
    assert np.linalg.eigvalsh(g).min() >= -1e-9 * np.abs(g).max()


def test_eq1_frame_layout_roi(oracle_mod):
    """A region read out of a larger frame equals the region cut out beforehand."""
    rng = np.random.default_rng(1)
    n, H, W = 40, 10, 24
    img = (rng.random((n, H, W)) < 0.4).astype(np.uint8)
    bits = synth.pack_bits_lsb(torch.from_numpy(img.reshape(n, H * W))).numpy()
    da = dict(bits=1, height=5, width=7, x0=3, y0=2, row_stride=W, frame_stride_bytes=H * W // 8)
    db = dict(bits=1, height=4, width=9, x0=13, y0=5, row_stride=W, frame_stride_bytes=H * W // 8)
    r = oracle_mod.correlate(bits, da, bits, db, n)
    A = img[:, 2:7, 3:10].reshape(n, -1).astype(np.int64)
    B = img[:, 5:9, 13:22].reshape(n, -1).astype(np.int64)
    assert np.array_equal(r["s_ab"], A.T @ B)
    assert np.array_equal(r["s_a"], A.sum(0))


def test_eq1_overflow_refused(oracle_mod):
    d = dict(bits=8, height=1, width=1, x0=0, y0=0, row_stride=1, frame_stride_bytes=1)
    fr = np.zeros(1, dtype=np.uint8)
    with pytest.raises(ValueError):
        # N^2 * 255^2 >= 2^63 for N = 2e7: the exact numerator is not guaranteed
        oracle_mod.correlate(np.broadcast_to(fr, (1,)), d, fr, d, 20_000_000)


# ----------------------------------------------------------------------------- closed forms

def _closed_form(acq):
    """Expected covariance of the detector outputs under the source model."""
    L_a, L_b, Pa, Pb, s_a, s_b = synth.model_maps(acq)
    S = acq.S
    bins_a = [np.flatnonzero(np.kron(Pa[y], Pa[x])) for y in range(acq.side_a) for x in range(acq.side_a)]
    bins_b = [np.flatnonzero(np.kron(Pb[y], Pb[x])) for y in range(acq.side_b) for x in range(acq.side_b)]
    if acq.counts == "poisson8":
        # Gaussian moment theorem: Cov(|F_u|^2, |G_v|^2) = |E F_u G_v^*|^2
        K = np.abs(L_a @ L_b.conj().T) ** 2
        return np.array([[s_a * s_b * K[np.ix_(ia, ib)].sum() for ib in bins_b] for ia in bins_a])
    # E exp(-E^H Q E) = 1/det(I + Q) for E ~ CN(0, I); by Sylvester a small determinant
    def p0(rows):
        W = rows
        return 1.0 / np.real(np.linalg.det(np.eye(W.shape[0]) + W @ W.conj().T))
    Wa = [np.sqrt(s_a) * L_a[ia] for ia in bins_a]
    Wb = [np.sqrt(s_b) * L_b[ib] for ib in bins_b]
    pa = np.array([p0(w) for w in Wa])
    pb = np.array([p0(w) for w in Wb])
    g = np.array([[p0(np.vstack([wa, wb])) - pa[i] * pb[j] for j, wb in enumerate(Wb)]
                  for i, wa in enumerate(Wa)])
    if acq.counts == "binomial255":
        g = g * 255.0 * 255.0
    return g


@pytest.mark.slow
@pytest.mark.parametrize("counts,mean,power", [("poisson8", 2.0, 10.0), ("bernoulli", 1.0, 4.5),
                                               ("binomial255", 0.3, 10.0)])
def test_eq1_closed_form_source_model(oracle_mod, counts, mean, power):
    acq = synth.Acquisition(4, 4, 40000, mean, counts, src_side=8, seed=21)
    n = acq.n_frames
    A, B, fr, lay = _frames(acq)
    r = oracle_mod.correlate(fr, lay["a"], fr, lay["b"], n)
    g_hat = r["gamma"]
    expect = (1.0 - 1.0 / n) * _closed_form(acq)
    ua = A.reshape(n, -1).double().numpy()
    ub = B.reshape(n, -1).double().numpy()
    va, vb = ua.var(0), ub.var(0)
    se = np.sqrt((va[:, None] * vb[None, :] + g_hat ** 2) / n)
    z = (g_hat - expect) / se
    # 256 entries: |z| beyond 5 has probability ~1e-4 under the model
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    assert abs(z.mean()) < 0.5
    # the structure is really there: correlations well above noise somewhere
    # (binary frames carry weaker correlations than counts)
    assert np.abs(expect / se).max() > power


@pytest.mark.slow
def test_eq1_independent_detectors_zero_mean(oracle_mod):
    """Frames of A and B drawn from independent sources: Gamma ~ 0 within noise."""
    acq = synth.Acquisition(4, 4, 20000, 2.0, "poisson8", src_side=8, seed=1)
    A, _ = synth.generate(acq, "cpu")
    _, B = synth.generate(synth.frames.replace(acq, seed=2), "cpu")
    fr, lay = synth.pack_side_by_side(A, B, 8)
    n = acq.n_frames
    r = oracle_mod.correlate(fr.numpy(), lay["a"], fr.numpy(), lay["b"], n)
    va = A.reshape(n, -1).double().var(0).numpy()
    vb = B.reshape(n, -1).double().var(0).numpy()
    z = r["gamma"] / np.sqrt(va[:, None] * vb[None, :] / n)
    assert np.abs(z).max() < 5.0
    assert abs(z.mean()) < 0.5


# ----------------------------------------------------------------------------- refocusing

def test_refocus_hand_worked(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "refocus_hand.json")))
    al = [p[0] for p in g["planes"]]
    be = [p[1] for p in g["planes"]]
    out = oracle_mod.refocus(np.array(g["gamma"], dtype=np.float64), g["ha"], g["wa"], g["hb"],
                             g["wb"], al, be)
    assert np.array_equal(out, np.array(g["out"]))


def _scipy_refocus(gamma, ha, wa, hb, wb, alpha, beta):
    from scipy import ndimage

    cxa, cya, cxb, cyb = (wa - 1) / 2, (ha - 1) / 2, (wb - 1) / 2, (hb - 1) / 2
    sx, sy = wa / wb, ha / hb
    out = np.zeros((len(alpha), ha, wa))
    rr, cc = np.meshgrid(np.arange(ha), np.arange(wa), indexing="ij")
    for p, (al, be) in enumerate(zip(alpha, beta)):
        for br in range(hb):
            for bc in range(wb):
                img = gamma[:, br * wb + bc].reshape(ha, wa)
                uy = al * (rr - cya) + be * sy * (br - cyb) + cya
                ux = al * (cc - cxa) + be * sx * (bc - cxb) + cxa
                out[p] += ndimage.map_coordinates(img, [uy, ux], order=1, mode="grid-constant",
                                                  cval=0.0, prefilter=False)
    return out


def test_refocus_matches_scipy_linear_interpolation(oracle_mod):
    rng = np.random.default_rng(7)
    ha, wa, hb, wb = 9, 12, 4, 6
    gamma = rng.standard_normal((ha * wa, hb * wb))
    alpha = np.array([0.5, 0.83, 1.0, 1.37, 1.5, 2.2])
    beta = np.array([0.5, 0.17, 0.0, -0.37, -0.5, 0.9])
    out = oracle_mod.refocus(gamma, ha, wa, hb, wb, alpha, beta)
    ref = _scipy_refocus(gamma, ha, wa, hb, wb, alpha, beta)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.abs(gamma).sum(1).max()


def test_refocus_focused_plane_is_row_sum(oracle_mod):
    rng = np.random.default_rng(8)
    ha, wa, hb, wb = 8, 8, 4, 4
    gamma = rng.integers(-1000, 1000, size=(ha * wa, hb * wb)).astype(np.float64)
    out = oracle_mod.refocus(gamma, ha, wa, hb, wb, [1.0], [0.0])
    assert np.array_equal(out[0].reshape(-1), gamma.sum(1))


def test_refocus_integer_shifts_are_gathers(oracle_mod):
    """alpha=1, beta=1, W_a/W_b=2, even W_b: every sample lands on a pixel."""
    rng = np.random.default_rng(9)
    ha, wa, hb, wb = 8, 8, 4, 4
    gamma = rng.integers(-50, 50, size=(ha * wa, hb * wb)).astype(np.float64)
    out = oracle_mod.refocus(gamma, ha, wa, hb, wb, [1.0], [1.0])
    want = np.zeros((ha, wa))
    for br in range(hb):
        for bc in range(wb):
            dy = int(round(2 * (br - (hb - 1) / 2)))
            dx = int(round(2 * (bc - (wb - 1) / 2)))
            img = gamma[:, br * wb + bc].reshape(ha, wa)
            for r in range(ha):
                for c in range(wa):
                    y, x = r + dy, c + dx
                    if 0 <= y < ha and 0 <= x < wa:
                        want[r, c] += img[y, x]
    assert np.array_equal(out[0], want)


def test_refocus_constant_gamma_counts_in_range_weight(oracle_mod):
    ha, wa, hb, wb = 6, 10, 3, 5
    gamma = np.ones((ha * wa, hb * wb))
    al, be = 1.3, -0.4
    out = oracle_mod.refocus(gamma, ha, wa, hb, wb, [al], [be])

    def wsum(u, n):  # total weight of the in-range taps of a 1-D linear interpolation
        f0 = np.floor(u)
        f = u - f0
        return (1 - f) * ((f0 >= 0) & (f0 < n)) + f * ((f0 + 1 >= 0) & (f0 + 1 < n))

    want = np.zeros((ha, wa))
    for br in range(hb):
        for bc in range(wb):
            uy = al * (np.arange(ha) - (ha - 1) / 2) + be * (ha / hb) * (br - (hb - 1) / 2) + (ha - 1) / 2
            ux = al * (np.arange(wa) - (wa - 1) / 2) + be * (wa / wb) * (bc - (wb - 1) / 2) + (wa - 1) / 2
            want += np.outer(wsum(uy, ha), wsum(ux, wa))
    assert np.max(np.abs(out[0] - want)) < 1e-12 * hb * wb


def test_refocus_linear(oracle_mod):
    rng = np.random.default_rng(10)
    ha, wa, hb, wb = 7, 5, 3, 3
    g1 = rng.standard_normal((ha * wa, hb * wb))
    g2 = rng.standard_normal((ha * wa, hb * wb))
    al, be = [0.7, 1.2], [0.3, -0.2]
    o1 = oracle_mod.refocus(g1, ha, wa, hb, wb, al, be)
    o2 = oracle_mod.refocus(g2, ha, wa, hb, wb, al, be)
    o12 = oracle_mod.refocus(g1 + 3.0 * g2, ha, wa, hb, wb, al, be)
    assert np.max(np.abs(o12 - (o1 + 3.0 * o2))) < 1e-12 * 4 * hb * wb * 4


def test_row_subset_equals_the_full_oracle_on_bin_layout_frames(oracle_mod):
    """oracle.correlate_rows (rows of outputs too large to hold whole) gives the
    same rows as the full computation, on frames in the layout of the paper's
    .bin files (two side-by-side images, LSB-first bits)."""
    import synth

    fr = synth.bin_file_frames(300, 1, height=16, width=64, p=0.2)
    lay = synth.bin_file_layout(16, 64)
    h = fr.numpy()
    full = oracle_mod.correlate(h, lay["a"], h, lay["b"], 300)
    part = oracle_mod.correlate_rows(h, lay["a"], h, lay["b"], 300, 100, 140)
    assert np.array_equal(full["s_ab"][100:140], part["s_ab"])
    assert np.array_equal(full["gamma"][100:140].view(np.int64), part["gamma"].view(np.int64))
    assert np.array_equal(full["s_a"], part["s_a"]) and np.array_equal(full["s_b"], part["s_b"])
    # the shared per-frame intensity makes every pixel pair correlated: Gamma = Var(p_i)
    assert abs(full["gamma"].mean() - (0.1 ** 2) / 3) < 5e-4


def _scipy_refocus4d(gamma, ha, wa, hb, wb, alpha, beta, gam, delta):
    """The 4-D refocusing written with scipy's N-D linear interpolation of the
    4-D array G[ya, xa, yb, xb] (grid-constant: 0 outside)."""
    from scipy import ndimage

    g4 = gamma.reshape(ha, wa, hb, wb)
    cxa, cya, cxb, cyb = (wa - 1) / 2, (ha - 1) / 2, (wb - 1) / 2, (hb - 1) / 2
    sx, sy = wa / wb, ha / hb
    rr, cc = np.meshgrid(np.arange(ha), np.arange(wa), indexing="ij")
    out = np.zeros((len(alpha), ha, wa))
    for p, (al, be, ga, de) in enumerate(zip(alpha, beta, gam, delta)):
        for jr in range(hb):
            for jc in range(wb):
                coords = [al * (rr - cya) + be * sy * (jr - cyb) + cya,
                          al * (cc - cxa) + be * sx * (jc - cxb) + cxa,
                          ga * (rr - cya) / sy + de * (jr - cyb) + cyb,
                          ga * (cc - cxa) / sx + de * (jc - cxb) + cxb]
                out[p] += ndimage.map_coordinates(g4, coords, order=1, mode="grid-constant", cval=0.0,
                                                  prefilter=False)
    return out


def test_refocus4d_matches_scipy_4d_linear_interpolation(oracle_mod):
    rng = np.random.default_rng(17)
    ha, wa, hb, wb = 7, 9, 4, 5
    gamma = rng.standard_normal((ha * wa, hb * wb))
    alpha = np.array([0.6, 1.0, 1.3, 0.9])
    beta = np.array([0.4, 0.0, -0.3, 0.25])
    gam = np.array([0.3, 0.0, -0.45, 0.7])
    delta = np.array([0.8, 1.0, 1.2, 0.5])
    out = oracle_mod.refocus4d(gamma, ha, wa, hb, wb, alpha, beta, gam, delta)
    ref = _scipy_refocus4d(gamma, ha, wa, hb, wb, alpha, beta, gam, delta)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.abs(gamma).sum(1).max()


def test_refocus4d_reduces_to_the_2d_refocusing(oracle_mod):
    """gamma = 0, delta = 1: the angular sample points are the angular pixels."""
    rng = np.random.default_rng(18)
    ha, wa, hb, wb = 8, 10, 4, 5
    gamma = rng.standard_normal((ha * wa, hb * wb))
    alpha = np.array([0.5, 1.0, 1.4])
    beta = 1.0 - alpha
    out4 = oracle_mod.refocus4d(gamma, ha, wa, hb, wb, alpha, beta, np.zeros(3), np.ones(3))
    out2 = oracle_mod.refocus(gamma, ha, wa, hb, wb, alpha, beta)
    assert np.max(np.abs(out4 - out2)) <= 1e-12 * np.abs(gamma).sum(1).max()
