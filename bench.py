"""Benchmark of the CPI hot path on GB300.

One step = one pass of the whole path over one acquisition of synthetic frames
already resident in HBM: ingest (transpose + marginal sums; bit-unpack for
binary frames), the raw-moment tensor-core contraction, the int64 fold + FP64
Gamma of Eq. (1), and refocusing into P planes.  Default workload: 128x128
spatial vs 64x64 angular uint8 counts (sums of 255 binary sub-frames),
N = 50000 frames side by side, 128 refocusing planes; the line also carries the
64x64 vs 32x32 binary workload, the batch of 64 uneven acquisitions and the
denoiser's frames saved under "workloads".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  `value` is the whole-step throughput in
int8-equivalent tera-operations per second, 2 * M_a * M_b * N / t_step, summed
over ranks for N > 1 (independent replicas, one per GPU: the correlation of one
acquisition needs no exchange between GPUs).  `--impl reference` times the CPU
oracle (plain C, OpenMP): the whole step, or for the default workload a
proportional sample of it (see ORACLE_SAMPLE_IMAGE_ROWS).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (acquisition key, planes)
    "spad_1bit": ("spad_1bit", 32),
    "small_u8": ("small_u8", 4),
    "large_u8": ("large_u8", 128),
    "batched": (None, 256),      # 64 uneven uint8 acquisitions, one batch call per step
    "denoise": (None, 0),        # learned denoiser: training, inference and frames saved
    "paper_scale": (None, 0),    # 256x256 vs 256x256 binary, .bin-file blocks, Gamma 65536 x 65536
    "refocus4d": (None, 0),      # 4-D multilinear refocusing at the paper's RoIs and plane counts
    "streaming": (None, 0),      # streamed acquisitions: sustained frames/s (also a key of the default line)
}
L2_FLUSH_BYTES = 512 << 20     # > 129 MB L2


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.device_index = device_index

    def __enter__(self):
        try:
            import torch

            uuid = str(torch.cuda.get_device_properties(self.device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist_init(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, work_per_rank: float, seconds: float):
    """Whole-job throughput of `world` independent replicas: the work all ranks
    did divided by the slowest rank's time (tera-units per second)."""
    t_max = _max_over_ranks(world, seconds)
    return world * work_per_rank / t_max / 1e12, t_max


# ----------------------------------------------------------------------------- CPU oracle leg
# Everything below that calls the oracle runs outside the GPU arm's timed region,
# on rank 0 only: the CPU baseline (and the reference arm, which is the same
# oracle step) and the error check of the GPU results against it.

# Sample of one oracle step per workload: None = the whole step (Gamma of every
# row, every plane); k = the Gamma rows of the first k rows of the spatial image
# (k * W_a of the M_a rows) and the same fraction of the planes, so that the
# sample holds the correlation and refocusing work of the step in proportion.
ORACLE_SAMPLE_IMAGE_ROWS = {"small_u8": None, "spad_1bit": None, "large_u8": 1}


def oracle_step(acq, planes, frames_host, lay, image_rows, gamma_refocus=None):
    """One step (or its proportional sample) of the CPU oracle on the workload's
    frames: Eq. (1) then refocusing.  Returns (seconds, ops of the sample,
    description, oracle result of the correlation, refocused planes)."""
    import oracle

    oracle.build()
    la, lb = lay["a"], lay["b"]
    ha, wa, hb, wb = la["height"], la["width"], lb["height"], lb["width"]
    alpha, beta = planes
    P = len(alpha)
    n = acq.n_frames
    if image_rows is None:
        t0 = time.perf_counter()
        r = oracle.correlate(frames_host, la, frames_host, lb, n)
        ref = oracle.refocus(r["gamma"], ha, wa, hb, wb, alpha, beta)
        dt = time.perf_counter() - t0
        return dt, 2.0 * ha * wa * hb * wb * n, "the whole step: Eq. (1) for every entry, every plane", r, ref
    k = int(image_rows)
    q = max(1, round(P * k / ha))
    sub = dict(la, height=k)             # Gamma rows 0 .. k * wa - 1
    if gamma_refocus is None:
        gamma_refocus = synth_gamma(ha * wa, hb * wb)
    t0 = time.perf_counter()
    r = oracle.correlate(frames_host, sub, frames_host, lb, n)
    ref = oracle.refocus(gamma_refocus, ha, wa, hb, wb, alpha[:q], beta[:q])
    dt = time.perf_counter() - t0
    desc = (f"Eq. (1) for the Gamma rows of spatial image row(s) 0..{k - 1} ({k * wa} of {ha * wa} rows, all "
            f"{n} frames) and {q} of {P} planes (a seeded stand-in Gamma of the full shape): {k}/{ha} of "
            f"the step's correlation and refocusing work")
    return dt, 2.0 * k * wa * hb * wb * n, desc, r, ref


def synth_gamma(ma, mb, seed=20692):
    import synth

    return synth.random_gamma(ma, mb, seed)


def oracle_leg(workload, acq, planes, frames_host, lay, reps, cpi_refocus_fn, gpu_gamma_rows):
    """The CPU baseline (`reps` oracle steps or samples) and the error of the GPU
    results against the oracle: Gamma bit for bit on the rows the oracle computed
    (with S_a, S_b in full), refocusing against FP64 on sampled planes."""
    import numpy as np

    import oracle

    la, lb = lay["a"], lay["b"]
    ha, wa, hb, wb = la["height"], la["width"], lb["height"], lb["width"]
    ma, mb = ha * wa, hb * wb
    alpha, beta = planes
    P = len(alpha)
    k = ORACLE_SAMPLE_IMAGE_ROWS[workload]
    g_ref = synth_gamma(ma, mb) if k is not None else None
    times = []
    for _ in range(reps):
        dt, ops, desc, r, _ = oracle_step(acq, planes, frames_host, lay, k, g_ref)
        times.append(dt)
    t = statistics.median(times)
    cpu = {"value": ops / t / 1e12, "unit": "TOPS (int8-equivalent)", "cores": oracle.threads(), "kind": "oracle",
           "sample": desc, "s_per_sample": t, "samples_timed": reps}
    if k is not None:
        cpu["s_per_full_step_extrapolated"] = t * ha / k
    # ---------------------------------------------------------------- Gamma
    if k is None:
        rows = [(0, ma)]
    else:     # a block at the start and one at a seeded position
        blk = max(1, min(128, ma // 2))
        r0 = int(np.random.default_rng(7).integers(blk, ma - blk + 1))
        rows = [(0, blk), (r0, r0 + blk)]
    checked = mism = 0
    sums_exact = True
    for (r0, r1) in rows:
        if k is None:
            want = r
        else:
            want = oracle.correlate_rows(frames_host, la, frames_host, lb, acq.n_frames, r0, r1)
        got = gpu_gamma_rows(r0, r1)
        wg = want["gamma"] if k is not None else want["gamma"][r0:r1]
        ws_ab = want["s_ab"] if k is not None else want["s_ab"][r0:r1]
        mism += int((got["gamma"].view(np.int64) != wg.view(np.int64)).sum())
        mism += int((got["s_ab"] != ws_ab).sum())
        checked += wg.size
        sums_exact &= bool(np.array_equal(got["s_a"], want["s_a"]) and np.array_equal(got["s_b"], want["s_b"]))
    # ---------------------------------------------------------------- refocus
    if k is None:
        g64 = r["gamma"]
        src = "the oracle's FP64 Gamma of this acquisition (GPU: its FP32 rounding)"
        pidx = list(range(P))
    else:
        g64 = g_ref
        src = "a seeded stand-in Gamma of the full shape, standard normal values (GPU: the same FP32 values)"
        pidx = sorted({0, P // 2 - 1, P // 2, P - 1})
    out = cpi_refocus_fn(g64)                                  # GPU, all P planes, as the step runs it
    ref = oracle.refocus(g64, ha, wa, hb, wb, alpha[pidx], beta[pidx])
    ones = oracle.refocus(np.ones((ma, mb)), ha, wa, hb, wb, alpha[pidx], beta[pidx])
    err = np.abs(out[pidx] - ref)
    gmax = float(np.abs(g64).max())
    errors = {
        "gamma": {"entries_checked": int(checked), "mismatches": mism, "bit_exact": mism == 0 and sums_exact,
                  "rows": [list(x) for x in rows], "marginals_exact": sums_exact,
                  "against": "oracle int64 sums and exact-numerator FP64 Gamma"},
        "refocus": {"planes_checked": pidx, "max_abs_err_over_max_gamma": float(err.max() / gmax),
                    "max_err_over_max_gamma_times_weight": float((err / np.maximum(1e-6 * gmax * ones, 1e-300)).max()
                                                                 * 1e-6),
                    "target": "1e-6 (literal: max|R - R_fp64| / max|Gamma|)", "input": src,
                    "against": "oracle refocusing in FP64"},
    }
    return cpu, errors


# ----------------------------------------------------------------------------- GPU arm

def run_native(args, world, rank, local):
    line = measure_single(args, args.workload, world, rank, with_cpu=not args.no_cpu_baseline)
    if args.workload == "large_u8" and not args.no_extras:
        # the other configurations, each measured the same way, as extra keys
        extra = {}
        for name, fn in (("spad_1bit", lambda: measure_single(args, "spad_1bit", world, rank, with_cpu=False,
                                                              with_errors=True, light=True)),
                         ("batched", lambda: run_batched(args, world, rank)),
                         ("denoise", lambda: denoise_frames_saved(args, world, rank)),
                         ("streaming", lambda: stream_rates(args, world, rank)),
                         ("refocus2d", lambda: refocus2d_paper_rois(args, world, rank))):
            t0 = time.time()
            r = fn()
            if r is not None:
                r["wall_s"] = time.time() - t0
                extra[name] = r
        if line is not None:
            line["workloads"] = extra
    return line


def _dtype(bits):
    if bits == 1:
        return "u1 -> packed e2m1 tensor-core operands (kind::f8f6f4, exact fp32 partials), int64 sums, f64 Gamma, f32 refocus"
    return ("u8 -> bf16 tensor-core (exact fp32 segments below 2^24 added into uint32 every S frames, S certified from the "
            "recorded maxima), int64 sums, f64 Gamma, f32 refocus")


def measure_single(args, workload, world, rank, with_cpu=True, with_errors=True, light=False):
    """One single-acquisition workload: the timed step, its stage breakdown and
    rooflines, e2e through the C ABI, the graph-replayed step, and (rank 0, one
    GPU) the oracle leg: CPU baseline and errors against the oracle."""
    import torch

    import paper_2407_20692_gb300 as cpi
    import synth

    cpi.load()
    key, n_planes = WORKLOADS[workload]
    acq = synth.frames.replace(synth.CONFIGS[key], seed=1000 + rank)
    dev = torch.device("cuda", torch.cuda.current_device())
    t_gen = time.time()
    A, B = synth.generate(acq, dev)
    fr, lay = synth.pack_side_by_side(A, B, acq.bits)
    del A, B
    torch.cuda.synchronize()
    t_gen = time.time() - t_gen
    la, lb = lay["a"], lay["b"]
    ha, wa, hb, wb = la["height"], la["width"], lb["height"], lb["width"]
    ma, mb, n = ha * wa, hb * wb, acq.n_frames
    mk = lambda t, l: cpi.frames(t, l["bits"], l["height"], l["width"], l["x0"], l["y0"],
                                 l["row_stride"], l["frame_stride_bytes"])
    a, b = mk(fr, la), mk(fr, lb)
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, n), dtype=torch.uint8, device=dev)
    s_ab = torch.empty((ma, mb), dtype=torch.int64, device=dev)
    s_a = torch.empty(ma, dtype=torch.int64, device=dev)
    s_b = torch.empty(mb, dtype=torch.int64, device=dev)
    gamma = torch.empty((ma, mb), dtype=torch.float64, device=dev)
    g32 = torch.empty((mb, ma), dtype=torch.float32, device=dev)
    alpha, beta = synth.uniform_planes(n_planes)
    planes = cpi.plane_array(alpha, beta)
    rws = torch.empty(cpi.cpi_refocus_workspace_size(ha, wa, hb, wb, n_planes), dtype=torch.uint8, device=dev)
    out = torch.empty((n_planes, ha, wa), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        cpi.cpi_correlate_stage(cpi.CPI_STAGE_INGEST, a, b, n, 0, s_ab, s_a, s_b, gamma, g32, ws, stream)
        if ev:
            ev[1].record(stream)
        cpi.cpi_correlate_stage(cpi.CPI_STAGE_MOMENTS, a, b, n, 0, s_ab, s_a, s_b, gamma, g32, ws, stream)
        if ev:
            ev[2].record(stream)
        cpi.cpi_correlate_stage(cpi.CPI_STAGE_FOLD, a, b, n, 0, s_ab, s_a, s_b, gamma, g32, ws, stream)
        if ev:
            ev[3].record(stream)
        cpi.cpi_refocus(g32, ha, wa, hb, wb, planes, out, rws, stream)
        if ev:
            ev[4].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error during warm-up")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            step(evs[k])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    _barrier(world)
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error in the timed region")
    parts = [[ev[i].elapsed_time(ev[i + 1]) for i in range(4)] for ev in evs]
    step_ms = [sum(p) for p in parts]
    total_s = sum(step_ms) / 1e3
    ops = 2.0 * ma * mb * n
    value, total_s_max = replica_throughput(world, ops * args.steps, total_s)
    mean = lambda i: sum(p[i] for p in parts) / args.steps
    ingest_ms, moments_ms, fold_ms, refocus_ms = mean(0), mean(1), mean(2), mean(3)

    # ---------------------------------------------------------------- roofline
    roofs = rooflines(ma, mb, n, n_planes, acq.bits, dict(ingest=ingest_ms, moments=moments_ms,
                                                          fold=fold_ms, refocus=refocus_ms), workload)
    dominant = max(roofs, key=lambda k: roofs[k]["ms"])
    roof = dict(roofs[dominant])
    # ---------------------------------------------------------------- e2e through the C ABI
    e2e = e2e_run(args, cpi, fr, lay, n, stream, dev, planes, n_planes, ws, rws)
    e2e_value = world * ops / _max_over_ranks(world, e2e["s_per_step"]) / 1e12

    # ---------------------------------------------------------------- graph-replayed step
    # The same step as one cpi_batch_correlate call with a single item: captured
    # into a CUDA graph on first use and replayed (what a fixed-shape acquisition
    # loop calls; removes the per-launch host dispatch that bounds small shapes).
    graph_ms = graph_leg(args, cpi, dict(a=a, b=b, n_frames=n, s_ab=s_ab, s_a=s_a, s_b=s_b, gamma=gamma,
                                         gamma_f32=g32, planes=planes, refocus_out=out), flush, stream, dev)
    graph_ms = _max_over_ranks(world, graph_ms / 1e3) * 1e3

    # ---------------------------------------------------------------- oracle leg (rank 0, one GPU)
    # One last plain step so that the outputs checked below are the timed path's.
    step()
    torch.cuda.synchronize()
    cpu = errors = None
    if rank == 0 and world == 1 and (with_cpu or with_errors):
        host = fr.cpu().numpy()

        def gamma_rows(r0, r1):
            return {"gamma": gamma[r0:r1].cpu().numpy(), "s_ab": s_ab[r0:r1].cpu().numpy(),
                    "s_a": s_a.cpu().numpy(), "s_b": s_b.cpu().numpy()}

        def refocus_fn(g64):
            gg = torch.tensor(g64.T.astype("float32"), device=dev).contiguous()
            o = torch.empty((n_planes, ha, wa), dtype=torch.float32, device=dev)
            cpi.cpi_refocus(gg, ha, wa, hb, wb, planes, o, rws, stream)
            torch.cuda.synchronize()
            r = o.cpu().double().numpy()
            del gg, o
            return r

        cpu, errors = oracle_leg(workload, acq, (alpha, beta), host, lay, args.cpu_reps if with_cpu else 1,
                                 refocus_fn, gamma_rows)
        if not with_cpu:
            cpu = None

    if rank != 0:
        return None
    clocks = clk.summary()
    line = {
        "metric": "Gamma int8-equivalent TOPS per whole step (ingest + raw-moment GEMM + fold/FP64 "
                  "Gamma + refocus)",
        "value": value,
        "unit": "TOPS (int8-equivalent, 2*Ma*Mb*N per step)",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sum(step_ms) / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": _dtype(acq.bits),
        "data": "synthetic (seeded chaotic-light source model; stand-in for the SwissSPAD2 dataset)",
        "config": single_config(workload, acq, ha, wa, hb, wb, n_planes, world),
        "parts_ms": {"ingest": ingest_ms, "moments": moments_ms, "fold": fold_ms, "refocus": refocus_ms},
        "gamma_tops": ops / ((ingest_ms + moments_ms + fold_ms) / 1e3) / 1e12,
        "refocus_planes_per_s": n_planes / (refocus_ms / 1e3),
        "roofline": roof,
        "rooflines_all": roofs,
        "e2e": {"value": e2e_value, "unit": "TOPS (int8-equivalent)",
                "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                "ms_per_step": e2e["s_per_step"] * 1e3},
        "graph_replay": {"ms_per_step": graph_ms, "value": world * ops / (graph_ms / 1e3) / 1e12,
                         "unit": "TOPS (int8-equivalent)",
                         "call": "cpi_batch_correlate, one item, CPI_BATCH_GRAPH | CPI_BATCH_TUNE"},
        "gpu_launches": kernels_per_step(wa, n_planes) * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
        "input_generation_s": t_gen,
    }
    if errors is not None:
        line["errors"] = errors
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if light:
        for k in ("rooflines_all", "graph_replay"):
            line.pop(k, None)
    return line


def kernels_per_step(wa, n_planes):
    """Kernels one step launches: ingest, raw-moment GEMM, fold, then per chunk of
    up to 128 planes the x coordinate tables, the x stage and the y stage, plus
    one repack of Gamma when its rows are not 16-byte aligned for the staging
    copies (widths not a multiple of 4, or of 16 above 248)."""
    repack = (wa % 4 != 0) if wa <= 248 else (wa % 16 != 0)
    return 3 + 3 * -(-n_planes // 128) + (1 if repack else 0)


SM_COUNT = 152
SMEM_BYTES_PER_CLK = 128          # shared-memory load bandwidth per SM per clock


def _traffic(kernel_key, workload):
    """DRAM bytes per launch from the committed ncu summary, valid only for the
    workload it was captured on and while the kernel's source files are unchanged
    since the capture (else None)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    ent = table.get(f"{kernel_key}@{workload}")
    if not ent or ent.get("workload") != workload:
        return None
    h = hashlib.sha256()
    for rel in ent["sources"]:
        src = os.path.join(ROOT, rel)
        if not os.path.exists(src):
            return None
        h.update(open(src, "rb").read())
    if h.hexdigest() != ent["sha256"]:
        return None
    return ent["dram_bytes_per_launch"]


def single_config(workload, acq, ha, wa, hb, wb, n_planes, world):
    """The `config` object of a single-acquisition workload (both arms print it)."""
    return {"workload": f"{workload}: spatial {ha}x{wa} vs angular {hb}x{wb}, "
                        f"{'binary bit-packed' if acq.bits == 1 else 'uint8'} frames side by side, "
                        f"N={acq.n_frames}, {n_planes} refocus planes",
            "M_a": ha * wa, "M_b": hb * wb, "N": acq.n_frames, "planes": n_planes,
            "parallelism": f"replicas x{world}", "l2": "flushed (512 MiB write) between steps"}


def rooflines(ma, mb, n, n_planes, bits, ms, workload):
    """Roofline of each stage: algorithmic work per launch / measured time,
    against the measured peak of its bound (MEASURED_PEAKS.json)."""
    peaks, src = _peaks()
    ops = 2.0 * ma * mb * n
    out = {}
    if bits == 1:
        tc_peak, tc_src = 2.0 * peaks["bf16_tflops"], f"{src} bf16 burst x 2 (nominal f8f6f4/BF16 dense ratio)"
        kname = "moments (tcgen05 kind::f8f6f4, E2M1 0/1 operands)"
    else:
        tc_peak, tc_src = peaks["bf16_tflops"], f"{src} bf16 burst"
        kname = "moments (tcgen05 kind::f16, BF16 integer operands)"
    a = ops / (ms["moments"] / 1e3) / 1e12
    out["moments"] = {"kernel": kname, "bound": "tensor", "achieved": a, "peak": tc_peak,
                      "unit": "TFLOP/s", "frac": a / tc_peak, "traffic": _traffic("moments", workload),
                      "peak_source": tc_src, "ms": ms["moments"],
                      "work": "2*Ma*Mb*N int8-equivalent ops"}
    kpad = (n + 255) // 256 * 256 if bits == 1 else (n + 127) // 128 * 128
    ing = (ma + mb) * n * bits / 8 + (ma + mb) * kpad * (0.5 if bits == 1 else 2)   # E2M1 half a byte, BF16 2
    a = ing / (ms["ingest"] / 1e3) / 1e9
    out["ingest"] = {"kernel": "ingest (frames -> K-major operands, marginals)", "bound": "hbm",
                     "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
                     "traffic": _traffic("ingest", workload), "peak_source": f"{src} hbm copy", "ms": ms["ingest"],
                     "work": "frame bytes read + operand bytes written"}
    fb = ma * mb * (4 + 8 + 8 + 4)
    a = fb / (ms["fold"] / 1e3) / 1e9
    out["fold"] = {"kernel": "fold (int64 S_ab, FP64 Gamma, FP32 slice-major copy)", "bound": "hbm",
                   "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
                   "traffic": _traffic("fold", workload), "peak_source": f"{src} hbm copy", "ms": ms["fold"],
                   "work": "24 B per Gamma entry"}
    # Refocus, as the workload's metric defines it: per-plane Gamma FP32 traffic
    # (P planes x Ma x Mb x 4 B, what an unfused per-plane gather reads) per
    # second against the HBM copy peak.  The x stage stages each band of Gamma
    # rows once per block of 4 planes and is bound on chip by shared-memory
    # loads, given as "lsu" (8 B of loads per plane, row, column and angular
    # pixel: the two taps of one sample).
    eff = n_planes * ma * mb * 4.0 / (ms["refocus"] / 1e3) / 1e9
    smem = n_planes * ma * mb * 8.0
    smem_peak = SM_COUNT * SMEM_BYTES_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9
    a = smem / (ms["refocus"] / 1e3) / 1e9
    out["refocus"] = {"kernel": "refocus (row-band x stage, 4 planes per staged slice band, + y stage over angular rows)",
                      "bound": "hbm", "achieved": eff, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": eff / peaks["hbm_gbs"], "traffic": _traffic("refocus", workload),
                      "peak_source": f"{src} hbm copy", "ms": ms["refocus"],
                      "work": "P x Ma x Mb x 4 B (one FP32 Gamma read per plane)",
                      "lsu": {"achieved": a, "peak": smem_peak, "unit": "GB/s", "frac": a / smem_peak,
                              "peak_source": "derived: 152 SMs x 128 B/clk shared-memory loads x max SM clock",
                              "work": "8 B of shared-memory reads per (plane, row, column, angular pixel)"}}
    return out


def run_batched(args, world, rank):
    """64 acquisitions of uneven size (uint8 Poisson counts), 256 refocus planes
    each, as one batch call per step (grouped persistent GEMM launches replayed
    from a CUDA graph)."""
    import torch

    import paper_2407_20692_gb300 as cpi
    import synth

    cpi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n_planes = WORKLOADS["batched"][1]
    alpha, beta = synth.uniform_planes(n_planes)
    planes = cpi.plane_array(alpha, beta)
    entries, keep = [], []
    ops = 0.0
    for acq in synth.batched_acquisitions(64, seed=1234 + rank):
        A, B = synth.generate(acq, dev)
        fr, lay = synth.pack_side_by_side(A, B, 8)
        del A, B
        la, lb = lay["a"], lay["b"]
        ma, mb = la["height"] * la["width"], lb["height"] * lb["width"]
        mk = lambda l: cpi.frames(fr, l["bits"], l["height"], l["width"], l["x0"], l["y0"],
                                  l["row_stride"], l["frame_stride_bytes"])
        e = dict(a=mk(la), b=mk(lb), n_frames=acq.n_frames,
                 s_ab=torch.empty((ma, mb), dtype=torch.int64, device=dev),
                 s_a=torch.empty(ma, dtype=torch.int64, device=dev),
                 s_b=torch.empty(mb, dtype=torch.int64, device=dev),
                 gamma=torch.empty((ma, mb), dtype=torch.float64, device=dev),
                 gamma_f32=torch.empty((mb, ma), dtype=torch.float32, device=dev),
                 planes=planes,
                 refocus_out=torch.empty((n_planes, la["height"], la["width"]), dtype=torch.float32, device=dev))
        entries.append(e)
        keep.append(fr)
        ops += 2.0 * ma * mb * acq.n_frames
    items = cpi.batch_items(entries)
    ws = torch.empty(cpi.cpi_batch_workspace_size(items), dtype=torch.uint8, device=dev)
    # correlation-only batch (same buffers), for the Gamma share of the step
    corr = [dict(e, planes=None, refocus_out=None) for e in entries]
    items_c = cpi.batch_items(corr)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.zero_()
        cpi.cpi_batch_correlate(items, ws, stream=stream)
        cpi.cpi_batch_correlate(items_c, ws, stream=stream)
    torch.cuda.synchronize()
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error during warm-up")

    def timed(it):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            cpi.cpi_batch_correlate(it, ws, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        step_ms = timed(items)
    corr_ms = timed(items_c)
    _barrier(world)
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error in the timed region")
    value, _ = replica_throughput(world, ops * args.steps, sum(step_ms) / 1e3)
    if rank != 0:
        return None
    peaks, src = _peaks()
    g_ms = sum(corr_ms) / len(corr_ms)
    a = ops / (g_ms / 1e3) / 1e12
    return {
        "metric": "Gamma int8-equivalent TOPS per whole step (ingest + raw-moment GEMM + fold/FP64 "
                  "Gamma + refocus) over a batch of 64 acquisitions",
        "value": value, "unit": "TOPS (int8-equivalent, sum of 2*Ma*Mb*N per step)", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype(8),
        "data": "synthetic (seeded chaotic-light source model)",
        "config": {"workload": "batched: 64 acquisitions, side_a ~ U{32..96}, side_b ~ U{16..48}, "
                               "N ~ U{5000..40000}, uint8 Poisson counts (mean 1-4), 256 planes each",
                   "ops_per_step": ops, "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MiB write) between steps"},
        "parts_ms": {"correlate_batch": g_ms, "refocus_batch": sum(step_ms) / len(step_ms) - g_ms},
        "gamma_tops": a,
        "refocus_planes_per_s": 64 * n_planes / ((sum(step_ms) / len(step_ms) - g_ms) / 1e3),
        "roofline": {"kernel": "correlation batch (ingest + grouped tcgen05 kind::f16 + fold), whole",
                     "bound": "tensor", "achieved": a, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": a / peaks["bf16_tflops"], "traffic": None,
                     "peak_source": f"{src} bf16 burst"},
        "gpu_launches": None, "clocks": clk.summary(),
    }


# Learned denoiser: 64x64 vs 32x32 uint8 Poisson counts (mean 2 photons), a
# seeded object per pair; inputs Gamma from N_in = 1000 frames, targets the
# closed-form expected Gamma; evaluated on held-out seeds against the plain Gamma.
DENOISE = dict(side_a=64, side_b=32, n_in=1000, mean=2.0, train_seeds=256, epochs=12, eval_seeds=6,
               n_eval=(1000, 2000, 5000, 10000, 20000, 50000), n_den=(1000, 2000, 5000), n_head=5000, lr=2e-3,
               planes=32)


def _denoise_acq(seed, n):
    import synth

    d = DENOISE
    return synth.Acquisition(d["side_a"], d["side_b"], n, d["mean"], "poisson8", seed=seed, mask_seed=seed)


def _gamma_prefixes(cpi, acq, dev, prefixes):
    """Gamma (float32, slice-major [Mb][Ma]) of the first k frames, for each k, through cpi_correlate."""
    import torch

    import synth

    A, B = synth.generate(acq, dev)
    fr, lay = synth.pack_side_by_side(A, B, 8)
    del A, B
    la, lb = lay["a"], lay["b"]
    mk = lambda l: cpi.frames(fr, 8, l["height"], l["width"], l["x0"], l["y0"], l["row_stride"],
                              l["frame_stride_bytes"])
    a, b = mk(la), mk(lb)
    ma, mb = la["height"] * la["width"], lb["height"] * lb["width"]
    s_ab = torch.empty((ma, mb), dtype=torch.int64, device=dev)
    s_a = torch.empty(ma, dtype=torch.int64, device=dev)
    s_b = torch.empty(mb, dtype=torch.int64, device=dev)
    g64 = torch.empty((ma, mb), dtype=torch.float64, device=dev)
    ws = torch.empty(cpi.cpi_correlate_workspace_size(a, b, max(prefixes)), dtype=torch.uint8, device=dev)
    out = []
    for k in prefixes:
        g32 = torch.empty((mb, ma), dtype=torch.float32, device=dev)
        cpi.cpi_correlate(a, b, k, s_ab, s_a, s_b, g64, g32, ws)
        out.append(g32)
    return out


def denoise_eval(cpi, model, dev, seeds):
    """Errors relative to the closed-form expected Gamma, of Gamma itself and of
    its refocused stack (32 uniform planes), on held-out seeds: the plain estimate
    at every N of DENOISE["n_eval"], the denoised one at DENOISE["n_den"], and
    the best scalar multiple of the plain estimate (uses the truth; shrinkage);
    zeros have relative error 1.  Frames saved: N_equiv / N_in with the plain
    error fitted as c / sqrt(N)."""
    import numpy as np
    import torch

    import synth

    d = DENOISE
    ha = wa = d["side_a"]
    hb = wb = d["side_b"]
    alpha, beta = synth.uniform_planes(d["planes"])
    planes = cpi.plane_array(alpha, beta)
    rws = torch.empty(cpi.cpi_refocus_workspace_size(ha, wa, hb, wb, d["planes"]), dtype=torch.uint8, device=dev)
    wsi = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb), dtype=torch.uint8, device=dev)

    def refocused(g):
        r = torch.empty((d["planes"], ha, wa), dtype=torch.float32, device=dev)
        cpi.cpi_refocus(g, ha, wa, hb, wb, planes, r, rws)
        return r.double()

    def rel(x, ref):
        return float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))

    keys = ("plain", "denoised", "shrink")
    err = {k: {n: [] for n in d["n_eval"]} for k in keys}
    err_r = {k: {n: [] for n in d["n_eval"]} for k in keys}
    for seed in seeds:
        acq = _denoise_acq(seed, max(d["n_eval"]))
        ref = synth.expected_gamma_counts(acq, dev, n_frames=10 ** 12).t().contiguous().to(torch.float32)
        ref_d, ref_r = ref.double(), refocused(ref)
        for n, g in zip(d["n_eval"], _gamma_prefixes(cpi, acq, dev, list(d["n_eval"]))):
            gd = g.double()
            a = float((gd * ref_d).sum() / (gd * gd).sum())
            rg = refocused(g)
            ar = float((rg * ref_r).sum() / (rg * rg).sum())
            err["plain"][n].append(rel(gd, ref_d))
            err["shrink"][n].append(rel(a * gd, ref_d))
            err_r["plain"][n].append(rel(rg, ref_r))
            err_r["shrink"][n].append(rel(ar * rg, ref_r))
            if n in d["n_den"]:
                out = torch.empty_like(g)
                cpi.cpi_denoise(model, g, out, ha, wa, hb, wb, wsi)
                err["denoised"][n].append(rel(out.double(), ref_d))
                err_r["denoised"][n].append(rel(refocused(out), ref_r))
    mean = lambda e: {k: {n: float(np.mean(v)) for n, v in e[k].items() if v} for k in keys}
    E, ER = mean(err), mean(err_r)

    def fit_c(ep):   # plain error = c / sqrt(N)
        return math.exp(float(np.mean([math.log(ep[n]) + 0.5 * math.log(n) for n in ep])))

    c, cr = fit_c(E["plain"]), fit_c(ER["plain"])
    n_equiv = {n: (c / E["denoised"][n]) ** 2 for n in d["n_den"]}
    n_equiv_r = {n: (cr / ER["denoised"][n]) ** 2 for n in d["n_den"]}
    return {"E": E, "ER": ER, "c": c, "cr": cr, "n_equiv": n_equiv, "n_equiv_r": n_equiv_r, "keys": keys,
            "saved": {n: n_equiv[n] / n for n in d["n_den"]}, "saved_r": {n: n_equiv_r[n] / n for n in d["n_den"]}}


COMMITTED_MODEL = os.path.join(ROOT, "paper_2407_20692_gb300", "models", "denoiser_64x64_32x32_n1000.npy")


def denoise_frames_saved(args, world, rank):
    """Frames saved by the committed denoiser (trained by `--workload denoise`) on
    held-out seeds, and its inference time per Gamma: the denoiser term of the
    headline metric without retraining."""
    import numpy as np
    import torch

    import paper_2407_20692_gb300 as cpi

    cpi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    d = DENOISE
    ha = wa = d["side_a"]
    hb = wb = d["side_b"]
    model = torch.tensor(np.load(COMMITTED_MODEL), device=dev)
    seeds = [100000 + 500000 + j for j in range(d["eval_seeds"])]        # held out from training
    ev = denoise_eval(cpi, model, dev, seeds)
    probe = _gamma_prefixes(cpi, _denoise_acq(seeds[0], d["n_in"]), dev, [d["n_in"]])[0]
    out = torch.empty_like(probe)
    wsi = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb), dtype=torch.uint8, device=dev)
    for _ in range(3):
        cpi.cpi_denoise(model, probe, out, ha, wa, hb, wb, wsi)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(10):
        cpi.cpi_denoise(model, probe, out, ha, wa, hb, wb, wsi)
    e1.record()
    torch.cuda.synchronize()
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error in the denoiser evaluation")
    if rank != 0:
        return None
    return {"metric": "frames saved by the denoiser at equal error of the refocused stack (N_equiv / N_in)",
            "value": ev["saved_r"][d["n_head"]], "unit": "x", "n_in": d["n_head"],
            "model": os.path.relpath(COMMITTED_MODEL, ROOT), "eval_seeds": len(seeds),
            "frames_saved_refocused": {str(k): v for k, v in ev["saved_r"].items()},
            "frames_saved_gamma": {str(k): v for k, v in ev["saved"].items()},
            "refocused_error": {k: {str(n): v for n, v in ev["ER"][k].items()} for k in ev["keys"]},
            "infer_ms_per_gamma": e0.elapsed_time(e1) / 10}


def run_denoise(args, world, rank):
    """Train the denoiser on seeded pairs, then measure on held-out seeds how many
    frames of the plain method the denoised Gamma is worth (N_equiv / N_in, with
    the plain error fitted as c / sqrt(N)), and time training and inference."""
    import numpy as np
    import torch

    import paper_2407_20692_gb300 as cpi
    import synth

    cpi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    d = DENOISE
    ha = wa = d["side_a"]
    hb = wb = d["side_b"]
    n_train = d["train_seeds"] if args.denoise_train_seeds is None else args.denoise_train_seeds
    epochs = d["epochs"] if args.denoise_epochs is None else args.denoise_epochs
    seed0 = 100000 + 10000 * rank
    t0 = time.time()
    # ---------------------------------------------------------------- training pairs
    gin, gtg = [], []
    for i in range(n_train):
        acq = _denoise_acq(seed0 + i, d["n_in"])
        gin.append(_gamma_prefixes(cpi, acq, dev, [d["n_in"]])[0])
        e = synth.expected_gamma_counts(acq, dev, n_frames=10 ** 12)       # the N -> infinity limit
        gtg.append(e.t().contiguous().to(torch.float32))
    torch.cuda.synchronize()
    t_data = time.time() - t0
    # ---------------------------------------------------------------- training
    model = torch.tensor(synth.denoiser_init(seed0), device=dev)
    m = torch.zeros_like(model)
    v = torch.zeros_like(model)
    grad = torch.empty_like(model)
    n_steps = n_train * epochs
    losses = torch.empty(n_steps, dtype=torch.float32, device=dev)
    ws = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb, training=True), dtype=torch.uint8, device=dev)
    order = np.random.Generator(np.random.Philox(seed0)).permutation(n_steps) % n_train
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for step in range(n_steps):
        i = int(order[step])
        lr = d["lr"] * (0.1 + 0.9 * 0.5 * (1.0 + math.cos(math.pi * step / n_steps)))   # cosine to lr / 10
        cpi.cpi_denoise_grad(model, gin[i], gtg[i], ha, wa, hb, wb, grad, losses[step:step + 1], ws)
        cpi.cpi_denoise_adam(model, m, v, grad, step + 1, lr)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error during training")
    lh = losses.cpu().numpy()
    del gin, gtg
    # ---------------------------------------------------------------- inference timing
    wsi = torch.empty(cpi.cpi_denoise_workspace_size(ha, wa, hb, wb), dtype=torch.uint8, device=dev)
    probe = _gamma_prefixes(cpi, _denoise_acq(seed0 + 999999, d["n_in"]), dev, [d["n_in"]])[0]
    out = torch.empty_like(probe)
    for _ in range(args.warmup):
        cpi.cpi_denoise(model, probe, out, ha, wa, hb, wb, wsi)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        cpi.cpi_denoise(model, probe, out, ha, wa, hb, wb, wsi)
    e1.record()
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1) / args.steps
    # ---------------------------------------------------------------- evaluation
    ev = denoise_eval(cpi, model, dev, [seed0 + 500000 + j for j in range(d["eval_seeds"])])
    E, ER, c, cr = ev["E"], ev["ER"], ev["c"], ev["cr"]
    n_equiv, n_equiv_r, saved, saved_r = ev["n_equiv"], ev["n_equiv_r"], ev["saved"], ev["saved_r"]
    keys = ev["keys"]
    if rank != 0:
        return None
    flops = 2.0 * hb * wb * ha * wa * 9 * (
        (9 * 32 + 32 * 32 + 32 * 32 + 32)          # forward
        + (32 + 32 * 32 + 32 * 32)                 # input gradients of layers 3, 2, 1
        + (9 * 32 + 32 * 32 + 32 * 32 + 32))       # weight gradients
    step_s = train_ms / 1e3 / n_steps
    ach = flops / step_s / 1e12
    # inference: the forward network on tcgen05 (widths 32/64/128), one Gamma
    fwd_flops = 2.0 * hb * wb * ha * wa * 9 * (9 * 32 + 32 * 32 + 32 * 32 + 32)
    tc_peak = _peaks()[0]["bf16_tflops"]
    fwd_ach = fwd_flops / (infer_ms / 1e3) / 1e12
    if args.save_model:
        np.save(args.save_model, model.cpu().numpy())
    return {
        "metric": "frames saved by the denoiser at equal error of the refocused stack "
                  f"(N_equiv / N_in at N_in = {d['n_head']}; model trained on Gamma from {d['n_in']} frames)",
        "value": saved_r[d["n_head"]], "unit": "x (frames of the plain method per input frame)", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": infer_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 activations and weights, fp32 accumulation",
        "data": "synthetic (seeded chaotic-light source, seeded object per pair; targets: closed-form expected Gamma)",
        "config": {"workload": f"denoise: spatial {ha}x{wa}, angular {hb}x{wb}, uint8 Poisson mean {d['mean']}, "
                               f"inputs Gamma from N = {d['n_in']}", "train_seeds": n_train, "epochs": epochs,
                   "eval_seeds": d["eval_seeds"], "parallelism": f"replicas x{world}"},
        "denoiser": {"gamma_error": {k: {str(n): v for n, v in E[k].items()} for k in keys},
                     "refocused_error": {k: {str(n): v for n, v in ER[k].items()} for k in keys},
                     "zeros_error": 1.0, "plain_fit_c": c, "plain_fit_c_refocused": cr,
                     "n_equiv": {str(k): v for k, v in n_equiv.items()},
                     "frames_saved": {str(k): v for k, v in saved.items()},
                     "n_equiv_refocused": {str(k): v for k, v in n_equiv_r.items()},
                     "frames_saved_refocused": {str(k): v for k, v in saved_r.items()},
                     "loss_first_last": [float(lh[:16].mean()), float(lh[-16:].mean())],
                     "train_ms_per_step": train_ms / n_steps, "infer_ms_per_gamma": infer_ms,
                     "data_s": t_data},
        "roofline": {"kernel": "denoiser inference (4 convolutions as tcgen05 implicit GEMMs, bf16 in, FP32 sums)",
                     "bound": "tensor", "achieved": fwd_ach, "peak": tc_peak, "unit": "TFLOP/s",
                     "frac": fwd_ach / tc_peak, "traffic": None, "peak_source": "measured bf16 burst",
                     "work": "forward network of one Gamma (1024 slices of 64 x 64; MMA padding not counted)"},
        "roofline_training": {"kernel": "denoiser training step (forward, hidden-layer input gradients and weight "
                                        "gradients on tcgen05, gradients as two bf16 terms; last layer's input "
                                        "gradient on the FP32 pipe)",
                              "bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s",
                              "frac": ach / tc_peak, "peak_source": "measured bf16 burst",
                              "work": "forward + input gradients + weight gradients of one Gamma (1024 slices), "
                                      "counted once (the two bf16 terms and MMA padding not counted)"},
        "gpu_launches": None,
    }


# Paper scale (Section 2 / Section 4.1): 256 x 512 binary frames (two 256 x 256
# images side by side), files of 512 frames, streamed in blocks of 64 files.
PAPER_SCALE = dict(files=256, frames_per_file=512, files_per_block=64, p=0.1)


def run_paper_scale(args, world, rank):
    """Eq. (1) at the paper's size: Gamma of 65536 x 65536 from N = 131072 frames,
    accumulated block by block (cpi_correlate_accumulate) and finalised in FP64.
    value: frames resident in HBM; e2e: each block copied from pinned host memory
    inside the timed region, Gamma not copied back (34 GB) but one row of it is."""
    import torch

    import paper_2407_20692_gb300 as cpi
    import synth

    cpi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    d = PAPER_SCALE
    fb = d["frames_per_file"] * d["files_per_block"]
    n = d["files"] * d["frames_per_file"]
    fr = synth.bin_file_frames(n, 2407 + rank, p=d["p"], device=dev)
    lay = synth.bin_file_layout()
    mk = lambda t, l: cpi.frames(t, 1, l["height"], l["width"], l["x0"], l["y0"], l["row_stride"],
                                 l["frame_stride_bytes"])
    ma = mb = 256 * 256
    s_ab = torch.empty((ma, mb), dtype=torch.int64, device=dev)
    s_a = torch.empty(ma, dtype=torch.int64, device=dev)
    s_b = torch.empty(mb, dtype=torch.int64, device=dev)
    gamma = torch.empty((ma, mb), dtype=torch.float64, device=dev)
    ws = torch.empty(cpi.cpi_correlate_workspace_size(mk(fr, lay["a"]), mk(fr, lay["b"]), fb),
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(src, staging=None):
        s_ab.zero_()
        s_a.zero_()
        s_b.zero_()
        for f0 in range(0, n, fb):
            blk = src[f0:f0 + fb]
            if staging is not None:
                staging.copy_(blk, non_blocking=True)
                blk = staging
            cpi.cpi_correlate_accumulate(mk(blk, lay["a"]), mk(blk, lay["b"]), blk.shape[0], s_ab, s_a, s_b, ws,
                                         stream=stream)
        cpi.cpi_correlate_finalize(s_ab, s_a, s_b, ma, mb, n, gamma, None, stream=stream)

    for _ in range(args.warmup):
        step(fr)
    torch.cuda.synchronize()
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error during warm-up")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for e0, e1 in evs:
            e0.record(stream)
            step(fr)
            e1.record(stream)
        torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    ops = 2.0 * ma * mb * n
    value, _ = replica_throughput(world, ops * args.steps, sum(ms) / 1e3)
    # e2e: blocks from pinned host memory, one Gamma row read back per step
    host = fr.cpu().pin_memory()
    staging = torch.empty((fb, fr.shape[1]), dtype=torch.uint8, device=dev)
    row = torch.empty(mb, dtype=torch.float64).pin_memory()
    step(host, staging)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(max(1, args.steps // 2)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(host, staging)
        row.copy_(gamma[12345], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error in the timed region")
    if rank != 0:
        return None
    peaks, src = _peaks()
    tc_peak = 2.0 * peaks["bf16_tflops"]
    a = ops / (sum(ms) / len(ms) / 1e3) / 1e12
    e2e = world * ops / (sum(e2e_ms) / len(e2e_ms) / 1e3) / 1e12
    return {
        "metric": "Gamma int8-equivalent TOPS at paper scale: 256x256 vs 256x256 binary frames, N = 131072 "
                  "(256 files of 512 frames) in blocks of 64 files, int64 sums + FP64 Gamma of 65536 x 65536",
        "value": value, "unit": "TOPS (int8-equivalent, 2*Ma*Mb*N per step)", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u1 -> packed e2m1 tensor-core operands (kind::f8f6f4, exact fp32 partials), int64 sums, f64 Gamma",
        "data": "synthetic (.bin-layout binary frames, Bernoulli with a shared per-frame intensity)",
        "config": {"workload": "paper_scale", "M_a": ma, "M_b": mb, "N": n, "block_frames": fb,
                   "parallelism": f"replicas x{world}", "l2": "inputs (2.1 GB) and outputs larger than L2"},
        "e2e": {"value": e2e, "unit": "TOPS (int8-equivalent)", "h2d_bytes_per_step": int(fr.numel()),
                "d2h_bytes_per_step": mb * 8, "ms_per_step": sum(e2e_ms) / len(e2e_ms)},
        "roofline": {"kernel": "whole step (ingest + moments + fold per block, finalize)", "bound": "tensor",
                     "achieved": a, "peak": tc_peak, "unit": "TFLOP/s", "frac": a / tc_peak, "traffic": None,
                     "peak_source": f"{src} bf16 burst x 2 (nominal f8f6f4/BF16 dense ratio)"},
        "gpu_launches": None, "clocks": clk.summary(),
    }


# Streamed acquisitions (cpi_acq_*): blocks of frames pushed from pinned host
# memory while earlier blocks accumulate; sustained frames per second against a
# SPAD camera's ~10^5 binary frames per second (the paper's Section 1).
SPAD_FRAME_RATE = 1.0e5
STREAM_CASES = {
    "spad_1bit": dict(block=8192, blocks=12),       # 64x64 vs 32x32 binary frames, 768 B each
    "paper_roi": dict(block=32768, blocks=2),       # 256x256 vs 256x256 binary (.bin layout), 16 KiB each;
                                                    # blocks of 64 files of 512 frames (Section 4.1)
}


def stream_rates(args, world, rank):
    """Sustained frames/s of a streamed acquisition for each STREAM_CASES shape:
    wall time from the first cpi_acq_push to the finalised Gamma (FP32,
    slice-major) being ready."""
    import torch

    import paper_2407_20692_gb300 as cpi
    import synth

    cpi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    res = {}
    for name, c in STREAM_CASES.items():
        n = c["block"] * c["blocks"]
        if name == "spad_1bit":
            acq = synth.frames.replace(synth.CONFIGS["spad_1bit"], n_frames=n, seed=555 + rank)
            A, B = synth.generate(acq, dev)
            fr, lay = synth.pack_side_by_side(A, B, 1)
            del A, B
        else:
            fr = synth.bin_file_frames(n, 2407 + rank, p=0.1, device=dev)
            lay = synth.bin_file_layout()
        host = fr.cpu().pin_memory()
        mk = lambda l: cpi.frames(fr, 1, l["height"], l["width"], l["x0"], l["y0"], l["row_stride"],
                                  l["frame_stride_bytes"])
        a, b = mk(lay["a"]), mk(lay["b"])
        del fr
        ma = lay["a"]["height"] * lay["a"]["width"]
        mb = lay["b"]["height"] * lay["b"]["width"]
        s_ab = torch.empty((ma, mb), dtype=torch.int64, device=dev)
        s_a = torch.empty(ma, dtype=torch.int64, device=dev)
        s_b = torch.empty(mb, dtype=torch.int64, device=dev)
        g32 = torch.empty((mb, ma), dtype=torch.float32, device=dev)
        ws = torch.empty(cpi.cpi_acq_workspace_size(a, b, c["block"]), dtype=torch.uint8, device=dev)

        def run(nblocks):
            h = cpi.cpi_acq_begin(a, b, c["block"], s_ab, s_a, s_b, ws)
            for k in range(nblocks):
                cpi.cpi_acq_push(h, host[k * c["block"]:(k + 1) * c["block"]], c["block"])
            cpi.cpi_acq_finalize(h, None, g32)
            cpi.cpi_acq_end(h)

        run(1)                                    # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(c["blocks"])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if cpi.cpi_device_status() != 0:
            raise RuntimeError("device status error in the streaming leg")
        fps = n / _max_over_ranks(world, dt) * world
        res[name] = {"frames": n, "block_frames": c["block"], "frame_bytes": int(host.shape[1]),
                     "seconds": dt, "frames_per_s": fps, "vs_spad_rate": fps / SPAD_FRAME_RATE,
                     "tops": 2.0 * ma * mb * n / dt / 1e12,
                     "M_a": ma, "M_b": mb}
        del s_ab, s_a, s_b, g32, ws, host
        torch.cuda.empty_cache()
    if rank != 0:
        return None
    return {"metric": "sustained frames/s of a streamed acquisition (blocks pushed from pinned host memory "
                      "while earlier blocks accumulate; Gamma finalised at the end)",
            "spad_frame_rate": SPAD_FRAME_RATE, "cases": res}


def refocus2d_paper_rois(args, world, rank):
    """2-D refocusing (cpi_refocus) at the RoIs and plane counts of the paper's
    refocusing benchmark (Section 4.2): 128x128 vs 128x128 (Gamma 16384 x 16384)
    with 100 and 261 planes, and 256x256 vs 256x256 (Gamma 65536 x 65536, 17 GB
    FP32) with 100 planes.  Gamma is a seeded random FP32 array (the kernels'
    cost does not depend on its values); uniformly spaced planes."""
    import torch

    import paper_2407_20692_gb300 as cpi
    import synth

    cpi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    res = {}
    peaks, _ = _peaks()
    for side, P in ((128, 100), (128, 261), (256, 100)):
        M = side * side
        gen = torch.Generator(device=dev)
        gen.manual_seed(2692 + side)
        g32 = torch.randn((M, M), generator=gen, device=dev, dtype=torch.float32)
        alpha, beta = synth.uniform_planes(P)
        planes = cpi.plane_array(alpha, beta)
        out = torch.empty((P, side, side), dtype=torch.float32, device=dev)
        ws = torch.empty(cpi.cpi_refocus_workspace_size(side, side, side, side, P), dtype=torch.uint8, device=dev)
        cpi.cpi_refocus(g32, side, side, side, side, planes, out, ws)
        torch.cuda.synchronize()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            cpi.cpi_refocus(g32, side, side, side, side, planes, out, ws)
        e1.record()
        torch.cuda.synchronize()
        if cpi.cpi_device_status() != 0:
            raise RuntimeError("device status error")
        ms = e0.elapsed_time(e1) / reps
        samples = P * M * M
        res[f"{side}x{side}_P{P}"] = {
            "ms": ms, "planes_per_s": P / (ms / 1e3),
            "per_plane_gamma_gbs": samples * 4 / (ms / 1e3) / 1e9,
            "lsu_frac": samples * 8 / (ms / 1e3) / (SM_COUNT * SMEM_BYTES_PER_CLK *
                                                    peaks.get("sm_max_mhz", 2070.0) * 1e6)}
        del g32, ws, out
        torch.cuda.empty_cache()
    if rank != 0:
        return None
    return {"metric": "2-D refocusing planes/s at the paper's refocusing RoIs (seeded random Gamma)", "cases": res}


def refocus4d_planes(P):
    """Plane coefficients of the 4-D refocusing workload: alpha uniform in
    [0.5, 1.5], beta = 1 - alpha, gamma = (alpha - 1) / 2, delta = 1 - gamma."""
    import numpy as np

    a = np.linspace(0.5, 1.5, P) if P > 1 else np.array([1.0])
    g = 0.5 * (a - 1.0)
    return a, 1.0 - a, g, 1.0 - g


def run_refocus4d(args, world, rank):
    """4-D multilinear refocusing (Section 4.1) of a 128x128 vs 128x128 Gamma
    (16384 x 16384) for 100, 261 and 1000 planes and of a 256x256 vs 256x256 Gamma
    (65536 x 65536) for 100 planes (the RoIs and plane counts of the paper's
    refocusing benchmark).  Gamma is synthetic FP32 (the kernels' cost does not
    depend on its values)."""
    import numpy as np
    import torch

    import paper_2407_20692_gb300 as cpi

    cpi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    cases = [(128, 100), (128, 261), (128, 1000), (256, 100)]
    if args.r4_side:
        cases = [(args.r4_side, args.r4_planes)]
    res = {}
    for side, P in cases:
        ha = wa = hb = wb = side
        M = side * side
        gen = torch.Generator(device=dev)
        gen.manual_seed(4207 + side)
        g32 = torch.randn((M, M), generator=gen, device=dev, dtype=torch.float32)
        planes = cpi.plane4_array(*refocus4d_planes(P))
        out = torch.empty((P, ha, wa), dtype=torch.float32, device=dev)
        ws = torch.empty(cpi.cpi_refocus4d_workspace_size(ha, wa, hb, wb, P), dtype=torch.uint8, device=dev)
        reps = args.steps if args.r4_side else 3 if side == 128 else 1
        cpi.cpi_refocus4d(g32, ha, wa, hb, wb, planes, out, ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            cpi.cpi_refocus4d(g32, ha, wa, hb, wb, planes, out, ws)
        e1.record()
        torch.cuda.synchronize()
        if cpi.cpi_device_status() != 0:
            raise RuntimeError("device status error")
        ms = e0.elapsed_time(e1) / reps
        res[f"{side}x{side}_P{P}"] = {"ms": ms, "planes_per_s": P / (ms / 1e3),
                                      "per_plane_gamma_gbs": P * M * M * 4 / (ms / 1e3) / 1e9}
        del g32, ws, out
        torch.cuda.empty_cache()
    if rank != 0:
        return None
    head = res["128x128_P261"] if "128x128_P261" in res else next(iter(res.values()))
    peaks, src = _peaks()
    return {
        "metric": "4-D multilinear refocusing planes/s, 128x128 vs 128x128 Gamma (16384 x 16384), 261 planes",
        "value": head["planes_per_s"], "unit": "planes/s", "n_gpus": world,
        "steps": args.steps if args.r4_side else 3, "warmup": 1,
        "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 sums (compensated) over angular columns, f64 over angular rows",
        "data": "synthetic (random FP32 Gamma)",
        "config": {"workload": "refocus4d", "cases": list(res), "parallelism": f"replicas x{world}"},
        "cases": res,
        # As for the 2-D refocusing: per-plane Gamma FP32 traffic (what a per-plane
        # gather reads) against the HBM copy peak.  The column stage reads Gamma
        # from HBM once per 64 planes and is bound on chip (instruction issue and
        # shared-memory loads: 16 B of box loads per column-stage sample).
        "roofline": {"kernel": "4-D refocusing (column stage + double-float row stage)", "bound": "hbm",
                     "achieved": head["per_plane_gamma_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": head["per_plane_gamma_gbs"] / peaks["hbm_gbs"], "traffic": None,
                     "peak_source": f"{src} hbm copy",
                     "work": "P x Ma x Mb x 4 B (one FP32 Gamma read per plane)",
                     "lsu": {"achieved": head["per_plane_gamma_gbs"] * 4.0,
                             "peak": SM_COUNT * SMEM_BYTES_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9,
                             "unit": "GB/s",
                             "frac": head["per_plane_gamma_gbs"] * 4.0 / (
                                 SM_COUNT * SMEM_BYTES_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9),
                             "peak_source": "derived: 152 SMs x 128 B/clk shared-memory loads x max SM clock",
                             "work": "16 B of shared-memory box loads per (plane, spatial pixel, angular pixel)"}},
        "gpu_launches": None,
    }


def ws_row_bytes(n, bits):
    pad = 256 if bits == 1 else 128
    k = (n + pad - 1) // pad * pad
    return k * (1 if bits == 1 else 2)


def graph_leg(args, cpi, entry, flush, stream, dev):
    """Mean device time (ms) of the whole step as a graph-replayed single-item
    batch call, L2 flushed between steps (outside the timed pairs)."""
    import torch

    items = cpi.batch_items([entry])
    wsb = torch.empty(cpi.cpi_batch_workspace_size(items), dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        cpi.cpi_batch_correlate(items, wsb, stream=stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        cpi.cpi_batch_correlate(items, wsb, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    if cpi.cpi_device_status() != 0:
        raise RuntimeError("device status error in the graph-replayed leg")
    return sum(e0.elapsed_time(e1) for e0, e1 in evs) / len(evs)


def e2e_run(args, cpi, fr, lay, n, stream, dev, planes, n_planes, ws, rws):
    """Same step through the public API with host buffers: pinned frames copied
    in, Gamma (f64) and the refocused stack copied out, inside the timed region.
    As an acquisition loop would run it: frames, Gamma and the stack are
    double-buffered; step k's frames are copied in on an upload stream while step
    k - 1 computes, and its results are copied out on a download stream while
    step k refocuses and step k + 1 computes (step k + 2 waits for both before it
    reuses the buffers)."""
    import torch

    la, lb = lay["a"], lay["b"]
    ha, wa, hb, wb = la["height"], la["width"], lb["height"], lb["width"]
    ma, mb = ha * wa, hb * wb
    host_in = fr.cpu().pin_memory()
    dev_in = [torch.empty_like(fr) for _ in range(2)]
    s_ab = torch.empty((ma, mb), dtype=torch.int64, device=dev)
    s_a = torch.empty(ma, dtype=torch.int64, device=dev)
    s_b = torch.empty(mb, dtype=torch.int64, device=dev)
    g32 = torch.empty((mb, ma), dtype=torch.float32, device=dev)
    gamma = [torch.empty((ma, mb), dtype=torch.float64, device=dev) for _ in range(2)]
    out = [torch.empty((n_planes, ha, wa), dtype=torch.float32, device=dev) for _ in range(2)]
    host_g = [torch.empty((ma, mb), dtype=torch.float64).pin_memory() for _ in range(2)]
    host_o = [torch.empty((n_planes, ha, wa), dtype=torch.float32).pin_memory() for _ in range(2)]
    mk = lambda t, l: cpi.frames(t, l["bits"], l["height"], l["width"], l["x0"], l["y0"],
                                 l["row_stride"], l["frame_stride_bytes"])
    ab = [(mk(t, la), mk(t, lb)) for t in dev_in]
    copy = torch.cuda.Stream(device=dev)
    upload = torch.cuda.Stream(device=dev)
    done = [torch.cuda.Event(), torch.cuda.Event()]       # buffer i's copies out finished
    consumed = [torch.cuda.Event(), torch.cuda.Event()]   # frames buffer i read by its correlation
    arrived = [torch.cuda.Event(), torch.cuda.Event()]    # frames buffer i copied in
    for e in done:
        e.record(copy)
    for e in consumed:
        e.record(stream)

    def one(k):
        i = k % 2
        upload.wait_event(consumed[i])
        with torch.cuda.stream(upload):
            dev_in[i].copy_(host_in, non_blocking=True)
        arrived[i].record(upload)
        stream.wait_event(arrived[i])
        stream.wait_event(done[i])
        a, b = ab[i]
        cpi.cpi_correlate(a, b, n, s_ab, s_a, s_b, gamma[i], g32, ws, stream)
        consumed[i].record(stream)
        ready_g = torch.cuda.Event()
        ready_g.record(stream)
        cpi.cpi_refocus(g32, ha, wa, hb, wb, planes, out[i], rws, stream)
        ready_o = torch.cuda.Event()
        ready_o.record(stream)
        copy.wait_event(ready_g)
        with torch.cuda.stream(copy):
            host_g[i].copy_(gamma[i], non_blocking=True)
            copy.wait_event(ready_o)
            host_o[i].copy_(out[i], non_blocking=True)
        done[i].record(copy)

    for k in range(max(1, args.warmup)):
        one(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, args.steps)
    e0.record(stream)
    upload.wait_event(e0)          # every timed copy starts after e0
    for k in range(steps):
        one(k)
    stream.wait_event(done[(steps - 1) % 2])
    stream.wait_event(done[(steps - 2) % 2] if steps > 1 else done[0])
    e1.record(stream)
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3 / steps
    return {"s_per_step": s, "h2d": host_in.numel(),
            "d2h": host_g[0].numel() * 8 + host_o[0].numel() * 4}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    """The CPU oracle as it stands, one oracle step per timed step (rank 0 only):
    the whole step where it fits a few seconds (small_u8, spad_1bit), else a
    proportional sample of it (large_u8: ORACLE_SAMPLE_IMAGE_ROWS).  `steps` and
    `ms_per_step` are what was timed; `value` is the sample's own throughput."""
    if rank != 0:
        return None
    import torch

    import oracle
    import synth

    key, n_planes = WORKLOADS[args.workload]
    if key is None:
        return {"impl": "reference", "unavailable": "the oracle arm is defined for the single-acquisition "
                                                    "workloads (spad_1bit, small_u8, large_u8)"}
    acq = synth.frames.replace(synth.CONFIGS[key], seed=1000)
    A, B = synth.generate(acq, "cuda" if torch.cuda.is_available() else "cpu")
    fr, lay = synth.pack_side_by_side(A, B, acq.bits)
    del A, B
    host = fr.cpu().numpy()
    alpha, beta = synth.uniform_planes(n_planes)
    la, lb = lay["a"], lay["b"]
    ha, wa, hb, wb = la["height"], la["width"], lb["height"], lb["width"]
    k = ORACLE_SAMPLE_IMAGE_ROWS[args.workload]
    g_ref = synth_gamma(ha * wa, hb * wb) if k is not None else None
    for _ in range(args.warmup):
        oracle_step(acq, (alpha, beta), host, lay, k, g_ref)
    times = []
    ops = desc = None
    t_region = time.perf_counter()
    for _ in range(args.steps):
        t, ops, desc, _, _ = oracle_step(acq, (alpha, beta), host, lay, k, g_ref)
        times.append(t)
    t_region = time.perf_counter() - t_region
    s = sum(times) / len(times)
    value = ops / s / 1e12
    cpu = {"value": value, "unit": "TOPS (int8-equivalent)", "cores": oracle.threads(), "kind": "oracle",
           "sample": desc}
    line = {
        "impl": "reference",
        "metric": "Gamma int8-equivalent TOPS per whole step (ingest + raw-moment GEMM + fold/FP64 "
                  "Gamma + refocus)",
        "value": value, "unit": "TOPS (int8-equivalent, 2*Ma*Mb*N per step)", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/int64/f64 (CPU oracle)",
        "data": "synthetic (seeded chaotic-light source model)",
        "config": single_config(args.workload, acq, ha, wa, hb, wb, n_planes, world),
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "TOPS (int8-equivalent)", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s_timed_region": t_region,
    }
    if k is not None:
        line["sampled"] = {"fraction_of_step": k / ha,
                           "s_per_full_step_extrapolated": s * ha / k,
                           "note": "each timed step is the proportional sample described in cpu_baseline.sample; "
                                   "the full step is not run (extrapolated linearly, for context only)"}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large_u8")
    ap.add_argument("--cpu-reps", type=int, default=3, help="oracle steps (or samples) timed for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="large_u8: skip the other workloads' keys (spad_1bit, batched, denoise, streaming, "
                         "refocus2d)")
    ap.add_argument("--denoise-train-seeds", type=int, default=None)
    ap.add_argument("--denoise-epochs", type=int, default=None)
    ap.add_argument("--save-model", default=None)
    ap.add_argument("--r4-side", type=int, default=0, help="refocus4d: one case, side x side vs side x side")
    ap.add_argument("--r4-planes", type=int, default=64, help="refocus4d: planes of the --r4-side case")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = _dist_init(args)
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    elif args.workload == "batched":
        line = run_batched(args, world, rank)
    elif args.workload == "denoise":
        line = run_denoise(args, world, rank)
    elif args.workload == "paper_scale":
        line = run_paper_scale(args, world, rank)
    elif args.workload == "refocus4d":
        line = run_refocus4d(args, world, rank)
    elif args.workload == "streaming":
        line = stream_rates(args, world, rank)
    else:
        line = run_native(args, world, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
