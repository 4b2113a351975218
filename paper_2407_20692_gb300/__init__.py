"""Python binding of the GB300 correlation plenoptic imaging library (libcpi.so).

Argument marshalling only: every entry point below forwards to the function of
the same name in the C ABI (include/cpi.h) with raw device pointers taken from
torch tensors.  All computation happens in the library's CUDA kernels; there is
no fallback, and ``load()`` raises if the library cannot be built or loaded.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "CpiError", "load", "frames", "plane_array", "cpi_status_string", "cpi_abi_version",
    "cpi_correlate_workspace_size", "cpi_correlate", "cpi_correlate_accumulate",
    "cpi_correlate_finalize", "cpi_correlate_stage", "cpi_refocus_workspace_size", "cpi_refocus",
    "cpi_denoise", "cpi_device_status", "cpi_set_wait_timeout_ns", "cpi_selftest_wait_timeout",
    "CPI_STAGE_INGEST", "CPI_STAGE_MOMENTS", "CPI_STAGE_FOLD", "EXPORTED", "cpi_correlate_noalloc",
    "NOALLOC_SCRATCH_BYTES", "cpi_batch_item", "batch_items", "CPI_BATCH_GRAPH", "CPI_BATCH_TUNE", "CPI_BATCH_N128",
    "cpi_batch_workspace_size", "cpi_batch_correlate", "cpi_denoise_workspace_size", "cpi_denoise_grad",
    "cpi_denoise_adam", "DENOISER_PARAMS", "cpi_plane4", "plane4_array",
    "cpi_refocus4d_workspace_size", "cpi_refocus4d", "cpi_acq_workspace_size", "cpi_acq_begin", "cpi_acq_push",
    "cpi_acq_frames", "cpi_acq_finalize", "cpi_acq_sync", "cpi_acq_end",
]
CPI_BATCH_GRAPH, CPI_BATCH_TUNE, CPI_BATCH_N128 = 1, 2, 4
DENOISER_PARAMS = 21409

CPI_STAGE_INGEST, CPI_STAGE_MOMENTS, CPI_STAGE_FOLD = 1, 2, 3
STATUS = {0: "CPI_OK", 1: "CPI_ERR_INVALID_ARG", 2: "CPI_ERR_OVERFLOW", 3: "CPI_ERR_WORKSPACE",
          4: "CPI_ERR_UNSUPPORTED", 5: "CPI_ERR_CUDA", 6: "CPI_ERR_TIMEOUT"}

# Every symbol include/cpi.h declares.
EXPORTED = [
    "cpi_status_string", "cpi_abi_version", "cpi_correlate_workspace_size", "cpi_correlate",
    "cpi_correlate_accumulate", "cpi_correlate_finalize", "cpi_correlate_stage",
    "cpi_refocus_workspace_size", "cpi_refocus", "cpi_denoise", "cpi_device_status",
    "cpi_set_wait_timeout_ns", "cpi_selftest_wait_timeout", "cpi_correlate_noalloc",
    "cpi_batch_workspace_size", "cpi_batch_correlate", "cpi_denoise_workspace_size", "cpi_denoise_grad",
    "cpi_denoise_adam", "cpi_refocus4d_workspace_size", "cpi_refocus4d", "cpi_acq_workspace_size", "cpi_acq_begin",
    "cpi_acq_push", "cpi_acq_frames", "cpi_acq_finalize", "cpi_acq_sync", "cpi_acq_end",
]
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


class CpiError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class cpi_frames(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("bits", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("x0", ctypes.c_int32),
        ("y0", ctypes.c_int32),
        ("row_stride", ctypes.c_int64),
        ("frame_stride_bytes", ctypes.c_int64),
        ("bit_order", ctypes.c_int32),
    ]


class cpi_plane(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double)]


class cpi_plane4(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("delta", ctypes.c_double)]


class cpi_batch_item(ctypes.Structure):
    _fields_ = [
        ("a", cpi_frames),
        ("b", cpi_frames),
        ("n_frames", ctypes.c_int64),
        ("s_ab", ctypes.c_void_p),
        ("s_a", ctypes.c_void_p),
        ("s_b", ctypes.c_void_p),
        ("gamma", ctypes.c_void_p),
        ("gamma_f32", ctypes.c_void_p),
        ("planes", ctypes.POINTER(cpi_plane)),
        ("n_planes", ctypes.c_int32),
        ("refocus_out", ctypes.c_void_p),
    ]


_lib = None
_P = ctypes.c_void_p
_F = ctypes.POINTER(cpi_frames)


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libcpi.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found: {path}")
    lib = ctypes.CDLL(path)
    i32, i64, sz, st = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_int
    sig = {
        "cpi_status_string": ([st], ctypes.c_char_p),
        "cpi_abi_version": ([], i32),
        "cpi_correlate_workspace_size": ([_F, _F, i64], sz),
        "cpi_correlate": ([_F, _F, i64, _P, _P, _P, _P, _P, _P, sz, _P], st),
        "cpi_correlate_accumulate": ([_F, _F, i64, _P, _P, _P, _P, sz, _P], st),
        "cpi_correlate_finalize": ([_P, _P, _P, i64, i64, i64, _P, _P, _P], st),
        "cpi_correlate_stage": ([i32, _F, _F, i64, i32, _P, _P, _P, _P, _P, _P, sz, _P], st),
        "cpi_refocus_workspace_size": ([i32, i32, i32, i32, i32], sz),
        "cpi_refocus": ([_P, i32, i32, i32, i32, ctypes.POINTER(cpi_plane), i32, _P, _P, sz, _P], st),
        "cpi_denoise_workspace_size": ([i32, i32, i32, i32, i32], sz),
        "cpi_refocus4d_workspace_size": ([i32, i32, i32, i32, i32], sz),
        "cpi_refocus4d": ([_P, i32, i32, i32, i32, ctypes.POINTER(cpi_plane4), i32, _P, _P, sz, _P], st),
        "cpi_denoise": ([_P, _P, _P, i32, i32, i32, i32, _P, sz, _P], st),
        "cpi_denoise_grad": ([_P, _P, _P, i32, i32, i32, i32, _P, _P, _P, sz, _P], st),
        "cpi_denoise_adam": ([_P, _P, _P, _P, i64, ctypes.c_float, _P], st),
        "cpi_device_status": ([_P, i32], st),
        "cpi_set_wait_timeout_ns": ([i64], None),
        "cpi_selftest_wait_timeout": ([i64, _P], st),
        "cpi_correlate_noalloc": ([_F, _F, i64, _P, _P, _P, _P, _P, _P], st),
        "cpi_batch_workspace_size": ([ctypes.POINTER(cpi_batch_item), i32], sz),
        "cpi_batch_correlate": ([ctypes.POINTER(cpi_batch_item), i32, _P, sz, i32, _P], st),
        "cpi_acq_workspace_size": ([_F, _F, i64], sz),
        "cpi_acq_begin": ([ctypes.POINTER(_P), _F, _F, i64, _P, _P, _P, i64, _P, sz, _P], st),
        "cpi_acq_push": ([_P, _P, i64], st),
        "cpi_acq_frames": ([_P], i64),
        "cpi_acq_finalize": ([_P, _P, _P], st),
        "cpi_acq_sync": ([_P], st),
        "cpi_acq_end": ([_P], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


# ----------------------------------------------------------------------------- helpers

def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream)) if hasattr(stream, "cuda_stream") else ctypes.c_void_p(stream)


def _check(code: int, where: str):
    if code != 0:
        raise CpiError(code, where)


def frames(data, bits: int, height: int, width: int, x0: int = 0, y0: int = 0,
           row_stride: int | None = None, frame_stride_bytes: int | None = None,
           bit_order: int = 0) -> cpi_frames:
    """Descriptor of one detector region inside a frame buffer (a CUDA uint8 tensor
    or a raw device address)."""
    addr = data.data_ptr() if hasattr(data, "data_ptr") else int(data)
    rs = row_stride if row_stride is not None else width
    fs = frame_stride_bytes
    if fs is None:
        fs = height * rs if bits == 8 else (height * rs + 7) // 8
    return cpi_frames(addr, bits, height, width, x0, y0, rs, fs, bit_order)


def plane4_array(alpha, beta, gamma, delta):
    n = len(alpha)
    arr = (cpi_plane4 * n)()
    for i in range(n):
        arr[i].alpha, arr[i].beta = float(alpha[i]), float(beta[i])
        arr[i].gamma, arr[i].delta = float(gamma[i]), float(delta[i])
    return arr


def cpi_refocus4d_workspace_size(ha, wa, hb, wb, n_planes) -> int:
    return load().cpi_refocus4d_workspace_size(ha, wa, hb, wb, n_planes)


def cpi_refocus4d(gamma_f32, ha, wa, hb, wb, planes, out, workspace, stream=None):
    """planes: a ctypes array from plane4_array() (host memory)."""
    _check(load().cpi_refocus4d(_ptr(gamma_f32), ha, wa, hb, wb, planes, len(planes), _ptr(out), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)), "cpi_refocus4d")


def plane_array(alpha, beta):
    n = len(alpha)
    arr = (cpi_plane * n)()
    for i in range(n):
        arr[i].alpha = float(alpha[i])
        arr[i].beta = float(beta[i])
    return arr


# ----------------------------------------------------------------------------- entry points

def cpi_status_string(code: int) -> str:
    return load().cpi_status_string(code).decode()


def cpi_abi_version() -> int:
    return load().cpi_abi_version()


def cpi_correlate_workspace_size(a: cpi_frames, b: cpi_frames, n_frames: int) -> int:
    return load().cpi_correlate_workspace_size(ctypes.byref(a), ctypes.byref(b), n_frames)


def cpi_correlate(a, b, n_frames, s_ab, s_a, s_b, gamma, gamma_f32, workspace, stream=None):
    _check(load().cpi_correlate(ctypes.byref(a), ctypes.byref(b), n_frames, _ptr(s_ab), _ptr(s_a),
                                _ptr(s_b), _ptr(gamma), _ptr(gamma_f32), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)),
           "cpi_correlate")


def cpi_correlate_accumulate(a, b, n_frames, s_ab, s_a, s_b, workspace, stream=None):
    _check(load().cpi_correlate_accumulate(ctypes.byref(a), ctypes.byref(b), n_frames, _ptr(s_ab),
                                           _ptr(s_a), _ptr(s_b), _ptr(workspace),
                                           workspace.numel() * workspace.element_size(),
                                           _stream(stream)), "cpi_correlate_accumulate")


def cpi_correlate_finalize(s_ab, s_a, s_b, m_a, m_b, n_total, gamma, gamma_f32, stream=None):
    _check(load().cpi_correlate_finalize(_ptr(s_ab), _ptr(s_a), _ptr(s_b), m_a, m_b, n_total,
                                         _ptr(gamma), _ptr(gamma_f32), _stream(stream)),
           "cpi_correlate_finalize")


def cpi_correlate_stage(stage, a, b, n_frames, accumulate, s_ab, s_a, s_b, gamma, gamma_f32,
                        workspace, stream=None):
    _check(load().cpi_correlate_stage(stage, ctypes.byref(a), ctypes.byref(b), n_frames,
                                      1 if accumulate else 0, _ptr(s_ab), _ptr(s_a), _ptr(s_b),
                                      _ptr(gamma), _ptr(gamma_f32), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), _stream(stream)),
           "cpi_correlate_stage")


def cpi_refocus_workspace_size(ha, wa, hb, wb, n_planes) -> int:
    return load().cpi_refocus_workspace_size(ha, wa, hb, wb, n_planes)


def cpi_refocus(gamma_f32, ha, wa, hb, wb, planes, out, workspace, stream=None):
    """planes: a ctypes array from plane_array() (host memory)."""
    _check(load().cpi_refocus(_ptr(gamma_f32), ha, wa, hb, wb, planes, len(planes), _ptr(out),
                              _ptr(workspace), workspace.numel() * workspace.element_size(),
                              _stream(stream)), "cpi_refocus")


def cpi_denoise_workspace_size(ha, wa, hb, wb, training=False) -> int:
    return load().cpi_denoise_workspace_size(ha, wa, hb, wb, 1 if training else 0)


def cpi_denoise(model, gamma_in, gamma_out, ha, wa, hb, wb, workspace, stream=None):
    """model: float32 device tensor [DENOISER_PARAMS]; gamma_in/out: float32 [hb*wb][ha*wa]."""
    _check(load().cpi_denoise(_ptr(model), _ptr(gamma_in), _ptr(gamma_out), ha, wa, hb, wb, _ptr(workspace),
                              workspace.numel() * workspace.element_size(), _stream(stream)), "cpi_denoise")


def cpi_denoise_grad(model, gamma_in, gamma_target, ha, wa, hb, wb, grad, loss, workspace, stream=None):
    _check(load().cpi_denoise_grad(_ptr(model), _ptr(gamma_in), _ptr(gamma_target), ha, wa, hb, wb, _ptr(grad),
                                   _ptr(loss), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                   _stream(stream)), "cpi_denoise_grad")


def cpi_denoise_adam(model, m, v, grad, step, lr, stream=None):
    _check(load().cpi_denoise_adam(_ptr(model), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr),
                                   _stream(stream)), "cpi_denoise_adam")


def cpi_device_status(stream=None, clear: bool = True) -> int:
    return load().cpi_device_status(_stream(stream), 1 if clear else 0)


def cpi_set_wait_timeout_ns(ns: int) -> None:
    load().cpi_set_wait_timeout_ns(int(ns))


def cpi_correlate_noalloc(a, b, n_frames, s_ab, s_a, s_b, gamma, gamma_f32, stream=None):
    """Correlation using the library's built-in scratch instead of a caller
    workspace, for callers that cannot allocate device memory (see include/cpi.h)."""
    _check(load().cpi_correlate_noalloc(ctypes.byref(a), ctypes.byref(b), n_frames, _ptr(s_ab),
                                        _ptr(s_a), _ptr(s_b), _ptr(gamma), _ptr(gamma_f32),
                                        _stream(stream)), "cpi_correlate_noalloc")


def batch_items(entries):
    """ctypes array of cpi_batch_item from dicts with keys a, b, n_frames, s_ab,
    s_a, s_b, gamma, gamma_f32 (tensors or None), planes (plane_array or None),
    refocus_out (tensor or None).  Keep `entries` alive while the array is used."""
    arr = (cpi_batch_item * len(entries))()
    for i, e in enumerate(entries):
        it = arr[i]
        it.a, it.b, it.n_frames = e["a"], e["b"], e["n_frames"]
        for k in ("s_ab", "s_a", "s_b", "gamma", "gamma_f32", "refocus_out"):
            t = e.get(k)
            setattr(it, k, None if t is None else t.data_ptr())
        pl = e.get("planes")
        it.planes = ctypes.cast(pl, ctypes.POINTER(cpi_plane)) if pl is not None else None
        it.n_planes = len(pl) if pl is not None else 0
    return arr


def cpi_batch_workspace_size(items) -> int:
    return load().cpi_batch_workspace_size(items, len(items))


def cpi_batch_correlate(items, workspace, flags=CPI_BATCH_GRAPH | CPI_BATCH_TUNE, stream=None):
    _check(load().cpi_batch_correlate(items, len(items), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), flags,
                                      _stream(stream)), "cpi_batch_correlate")


def cpi_selftest_wait_timeout(timeout_ns: int, stream=None):
    _check(load().cpi_selftest_wait_timeout(int(timeout_ns), _stream(stream)),
           "cpi_selftest_wait_timeout")


# ----------------------------------------------------------------------------- streamed acquisitions

def cpi_acq_workspace_size(a, b, block_frames) -> int:
    return load().cpi_acq_workspace_size(ctypes.byref(a), ctypes.byref(b), int(block_frames))


def cpi_acq_begin(a, b, block_frames, s_ab, s_a, s_b, workspace, frames_done=0, stream=None):
    """Opens a streamed acquisition (include/cpi.h); returns its handle."""
    h = ctypes.c_void_p()
    _check(load().cpi_acq_begin(ctypes.byref(h), ctypes.byref(a), ctypes.byref(b), int(block_frames), _ptr(s_ab),
                                _ptr(s_a), _ptr(s_b), int(frames_done), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)), "cpi_acq_begin")
    return h


def cpi_acq_push(h, host_frames, n_frames):
    """host_frames: a CPU tensor (pinned for an overlapped copy) or a host address."""
    addr = host_frames.data_ptr() if hasattr(host_frames, "data_ptr") else int(host_frames)
    _check(load().cpi_acq_push(h, ctypes.c_void_p(addr), int(n_frames)), "cpi_acq_push")


def cpi_acq_frames(h) -> int:
    return int(load().cpi_acq_frames(h))


def cpi_acq_finalize(h, gamma, gamma_f32):
    _check(load().cpi_acq_finalize(h, _ptr(gamma), _ptr(gamma_f32)), "cpi_acq_finalize")


def cpi_acq_sync(h):
    _check(load().cpi_acq_sync(h), "cpi_acq_sync")


def cpi_acq_end(h):
    _check(load().cpi_acq_end(h), "cpi_acq_end")
