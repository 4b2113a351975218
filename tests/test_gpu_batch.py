"""Batches: many uneven acquisitions (binary and counts) in grouped persistent
launches replayed from a CUDA graph must give, item by item, exactly what the
single-acquisition entry points give (which the other GPU tests pin to the
oracle), on the first call and on replays after the inputs change."""

import numpy as np
import pytest
import torch

import paper_2407_20692_gb300 as cpi
import synth
import oracle
from gpu_util import assert_exact, desc, oracle_correlate, refocus_errors

pytestmark = pytest.mark.gpu

SPECS = [(40, 20, 3000, "poisson8", 1.5), (33, 17, 1500, "poisson8", 3.0), (64, 32, 5000, "bernoulli", 0.3),
         (24, 12, 800, "bernoulli", 0.3), (96, 48, 2500, "poisson8", 1.0), (50, 30, 4100, "poisson8", 2.0),
         (32, 16, 700, "bernoulli", 0.5)]


@pytest.fixture(scope="module", autouse=True)
def _ready(cuda_ready, oracle_mod):
    yield


def _make(seed_base):
    items, keep = [], []
    for k, (sa, sb, n, counts, mu) in enumerate(SPECS):
        acq = synth.Acquisition(sa, sb, n, mu, counts, seed=seed_base + k)
        A, B = synth.generate(acq, "cuda")
        fr, lay = synth.pack_side_by_side(A, B, acq.bits)
        ma, mb = sa * sa, sb * sb
        alpha, beta = synth.uniform_planes(6)
        e = dict(a=desc(fr, lay["a"]), b=desc(fr, lay["b"]), n_frames=n,
                 s_ab=torch.empty((ma, mb), dtype=torch.int64, device="cuda"),
                 s_a=torch.empty(ma, dtype=torch.int64, device="cuda"),
                 s_b=torch.empty(mb, dtype=torch.int64, device="cuda"),
                 gamma=torch.empty((ma, mb), dtype=torch.float64, device="cuda"),
                 gamma_f32=torch.empty((mb, ma), dtype=torch.float32, device="cuda"),
                 planes=cpi.plane_array(alpha, beta),
                 refocus_out=torch.empty((6, sa, sa), dtype=torch.float32, device="cuda"))
        items.append(e)
        keep.append((fr, lay, acq))
    return items, keep


def _individual(e, lay):
    a, b, n = e["a"], e["b"], e["n_frames"]
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, n), dtype=torch.uint8, device="cuda")
    out = {k: torch.empty_like(e[k]) for k in ("s_ab", "s_a", "s_b", "gamma", "gamma_f32", "refocus_out")}
    cpi.cpi_correlate(a, b, n, out["s_ab"], out["s_a"], out["s_b"], out["gamma"], out["gamma_f32"], ws)
    ha, wa, hb, wb = lay["a"]["height"], lay["a"]["width"], lay["b"]["height"], lay["b"]["width"]
    rws = torch.empty(cpi.cpi_refocus_workspace_size(ha, wa, hb, wb, len(e["planes"])), dtype=torch.uint8,
                      device="cuda")
    cpi.cpi_refocus(out["gamma_f32"], ha, wa, hb, wb, e["planes"], out["refocus_out"], rws)
    return out


def _check(items, keep):
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    for e, (fr, lay, acq) in zip(items, keep):
        ref = _individual(e, lay)
        torch.cuda.synchronize()
        for k in ("s_ab", "s_a", "s_b", "gamma", "gamma_f32", "refocus_out"):
            assert torch.equal(ref[k], e[k]), (acq, k)


def test_batch_equals_individual_calls_and_replays():
    items, keep = _make(100)
    arr = cpi.batch_items(items)
    ws = torch.empty(cpi.cpi_batch_workspace_size(arr), dtype=torch.uint8, device="cuda")
    cpi.cpi_batch_correlate(arr, ws)                     # tunes, captures and replays
    _check(items, keep)
    # new frames in the same buffers: the cached graph must see them
    for k, (fr, lay, acq) in enumerate(keep):
        A, B = synth.generate(synth.frames.replace(acq, seed=acq.seed + 50), "cuda")
        fr2, _ = synth.pack_side_by_side(A, B, acq.bits)
        fr.copy_(fr2)
    cpi.cpi_batch_correlate(arr, ws)
    _check(items, keep)
    # without the graph and the tuner
    for e in items:
        e["s_ab"].zero_()
    cpi.cpi_batch_correlate(arr, ws, flags=0)
    _check(items, keep)
    # 128 x 128 output tiles (without the tuner), also captured and replayed
    for flags in (cpi.CPI_BATCH_N128, cpi.CPI_BATCH_N128 | cpi.CPI_BATCH_GRAPH):
        for e in items:
            e["s_ab"].zero_()
            e["gamma"].zero_()
        cpi.cpi_batch_correlate(arr, ws, flags=flags)
        _check(items, keep)


def test_batch_every_item_against_oracle():
    """Every item of a graph-replayed batch, Gamma and its refocused stack, against
    the oracle on the same frames (not against the library's own single calls):
    sums and Gamma bit for bit, the refocused stack within the refocusing
    tolerance of the FP64 oracle refocusing the oracle's Gamma."""
    items, keep = _make(300)
    arr = cpi.batch_items(items)
    ws = torch.empty(cpi.cpi_batch_workspace_size(arr), dtype=torch.uint8, device="cuda")
    cpi.cpi_batch_correlate(arr, ws)
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    alpha, beta = synth.uniform_planes(6)
    for e, (fr, lay, acq) in zip(items, keep):
        want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], acq.n_frames)
        got = {k: e[k].cpu() for k in ("s_ab", "s_a", "s_b", "gamma")}
        assert_exact(got, want)
        ha, wa, hb, wb = lay["a"]["height"], lay["a"]["width"], lay["b"]["height"], lay["b"]["width"]
        ref = oracle.refocus(want["gamma"], ha, wa, hb, wb, alpha, beta)
        out = e["refocus_out"].cpu().double().numpy()
        literal, per_w, tol = refocus_errors(out, ref, want["gamma"], ha, wa, hb, wb, alpha, beta)
        assert (np.abs(out - ref) <= tol).all(), (acq, per_w)
        if hb * wb <= 256:         # the literal reading where FP32 can meet it (test_gpu_refocus.check_literal)
            assert literal <= 1e-6, (acq, literal)


def test_batch_of_64_uneven_acquisitions_sampled_against_oracle():
    """The benchmark's batch itself: 64 acquisitions of uneven size
    (synth.batched_acquisitions(64, seed=1234)), 256 planes each, one
    graph-captured, tuned cpi_batch_correlate call.  The oracle checks a seeded
    sample: the four smallest items in full (sums, Gamma, and four refocused
    planes), and four more items on two blocks of rows (the first 64 and 32 from
    a seeded position) of S_ab and Gamma, with all of S_a and S_b."""
    acqs = synth.batched_acquisitions(64, seed=1234)
    alpha, beta = synth.uniform_planes(256)
    planes = cpi.plane_array(alpha, beta)
    entries, keep = [], []
    for acq in acqs:
        A, B = synth.generate(acq, "cuda")
        fr, lay = synth.pack_side_by_side(A, B, 8)
        del A, B
        ma, mb = acq.side_a ** 2, acq.side_b ** 2
        entries.append(dict(a=desc(fr, lay["a"]), b=desc(fr, lay["b"]), n_frames=acq.n_frames,
                            s_ab=torch.empty((ma, mb), dtype=torch.int64, device="cuda"),
                            s_a=torch.empty(ma, dtype=torch.int64, device="cuda"),
                            s_b=torch.empty(mb, dtype=torch.int64, device="cuda"),
                            gamma=torch.empty((ma, mb), dtype=torch.float64, device="cuda"),
                            gamma_f32=torch.empty((mb, ma), dtype=torch.float32, device="cuda"),
                            planes=planes,
                            refocus_out=torch.empty((256, acq.side_a, acq.side_a), dtype=torch.float32,
                                                    device="cuda")))
        keep.append((fr, lay, acq))
    arr = cpi.batch_items(entries)
    ws = torch.empty(cpi.cpi_batch_workspace_size(arr), dtype=torch.uint8, device="cuda")
    cpi.cpi_batch_correlate(arr, ws)
    cpi.cpi_batch_correlate(arr, ws)          # replay of the captured graph
    torch.cuda.synchronize()
    assert cpi.cpi_device_status() == 0
    mac = [a.side_a ** 2 * a.side_b ** 2 * a.n_frames for a in acqs]
    order = np.argsort(mac)
    small = [int(i) for i in order[:4]]
    rng = np.random.default_rng(1234)
    large = [int(i) for i in rng.choice(order[4:], 4, replace=False)]
    pidx = [0, 127, 128, 255]
    for i in small:
        e, (fr, lay, acq) = entries[i], keep[i]
        want = oracle_correlate(fr.cpu().numpy(), lay["a"], lay["b"], acq.n_frames)
        assert_exact({k: e[k].cpu() for k in ("s_ab", "s_a", "s_b", "gamma")}, want)
        ha, hb = acq.side_a, acq.side_b
        ref = oracle.refocus(want["gamma"], ha, ha, hb, hb, alpha[pidx], beta[pidx])
        out = e["refocus_out"][pidx].cpu().double().numpy()
        literal, per_w, tol = refocus_errors(out, ref, want["gamma"], ha, ha, hb, hb, alpha[pidx], beta[pidx])
        assert (np.abs(out - ref) <= tol).all(), (acq, per_w)
        if hb * hb <= 256:         # the literal reading where FP32 can meet it (test_gpu_refocus.check_literal)
            assert literal <= 1e-6, (acq, literal)
    for i in large:
        e, (fr, lay, acq) = entries[i], keep[i]
        host = fr.cpu().numpy()
        ma = acq.side_a ** 2
        r0 = int(rng.integers(64, ma - 32))
        rows = [(0, 64), (r0, r0 + 32)]
        for r0, r1 in rows:
            want = oracle.correlate_rows(host, lay["a"], host, lay["b"], acq.n_frames, r0, r1)
            assert np.array_equal(e["s_ab"][r0:r1].cpu().numpy(), want["s_ab"]), (acq, r0)
            assert np.array_equal(e["gamma"][r0:r1].cpu().numpy().view(np.int64), want["gamma"].view(np.int64)), \
                (acq, r0)
        assert np.array_equal(e["s_a"].cpu().numpy(), want["s_a"])
        assert np.array_equal(e["s_b"].cpu().numpy(), want["s_b"])


def test_batch_rejects_bad_items():
    items, keep = _make(500)
    items[2]["s_ab"] = None
    arr = cpi.batch_items(items)
    with pytest.raises(cpi.CpiError) as e:
        cpi.cpi_batch_correlate(arr, torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert e.value.code == 1


_TUNE_CHILD = r"""
import os, sys, json
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import torch
import paper_2407_20692_gb300 as cpi
from test_gpu_batch import _tune_batch
items, keep = _tune_batch()
arr = cpi.batch_items(items)
ws = torch.empty(cpi.cpi_batch_workspace_size(arr), dtype=torch.uint8, device="cuda")
cpi.cpi_batch_correlate(arr, ws, flags=cpi.CPI_BATCH_TUNE)
torch.cuda.synchronize()
print(json.dumps([int(e["s_ab"].sum()) for e in items]))
"""


def _tune_batch():
    """Three acquisitions of shapes no other test uses (a fresh tuner key)."""
    items, keep = [], []
    for k, (sa, sb, n) in enumerate([(27, 13, 1300), (19, 11, 900), (35, 21, 2100)]):
        acq = synth.Acquisition(sa, sb, n, 1.5, "poisson8", seed=4400 + k)
        A, B = synth.generate(acq, "cuda")
        fr, lay = synth.pack_side_by_side(A, B, 8)
        ma, mb = sa * sa, sb * sb
        items.append(dict(a=desc(fr, lay["a"]), b=desc(fr, lay["b"]), n_frames=n,
                          s_ab=torch.empty((ma, mb), dtype=torch.int64, device="cuda"),
                          s_a=torch.empty(ma, dtype=torch.int64, device="cuda"),
                          s_b=torch.empty(mb, dtype=torch.int64, device="cuda"),
                          gamma=None, gamma_f32=None, planes=None, refocus_out=None))
        keep.append(fr)
    return items, keep


def test_tuner_cache_file(tmp_path, monkeypatch):
    """CPI_TUNE_CACHE: the first tuned call of a batch shape appends one line
    (key, frame-chunk split, tile width); a second process with the same shapes
    reads it instead of timing again (the file keeps one line) and gets the same
    sums."""
    import json
    import os
    import subprocess
    import sys

    path = tmp_path / "tune.txt"
    monkeypatch.setenv("CPI_TUNE_CACHE", str(path))
    items, keep = _tune_batch()
    arr = cpi.batch_items(items)
    ws = torch.empty(cpi.cpi_batch_workspace_size(arr), dtype=torch.uint8, device="cuda")
    cpi.cpi_batch_correlate(arr, ws, flags=cpi.CPI_BATCH_TUNE)
    torch.cuda.synchronize()
    lines = path.read_text().split("\n")
    lines = [ln for ln in lines if ln.strip()]
    assert len(lines) == 1
    key, split, width = lines[0].split()
    assert int(key, 16) > 0 and int(split) in (1, 2, 4) and int(width) in (128, 256)
    want = [int(e["s_ab"].sum()) for e in items]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = _TUNE_CHILD.format(root=root, tests=os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, CPI_TUNE_CACHE=str(path)))
    assert r.returncode == 0, r.stderr[-2000:]
    assert json.loads(r.stdout.strip().splitlines()[-1]) == want
    assert len([ln for ln in path.read_text().split("\n") if ln.strip()]) == 1
