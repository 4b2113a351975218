"""Python access to the plain-C CPU oracle (``cpi_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the library.  ``build()``
compiles the C file into ``oracle/_build/liboracle.so`` with gcc.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpi_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (no FMA contraction, OpenMP); returns the .so path."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Frames(ctypes.Structure):
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


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        _lib.oracle_unpack.argtypes = [P(_Frames), ctypes.c_int64, ctypes.c_void_p]
        _lib.oracle_correlate.argtypes = [P(_Frames), P(_Frames), ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_refocus4d.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        _lib.oracle_refocus4d.restype = ctypes.c_int
        _lib.oracle_refocus.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        _lib.oracle_threads.restype = ctypes.c_int
    return _lib


def threads() -> int:
    return int(lib().oracle_threads())


def _desc(frames: np.ndarray, d: dict) -> _Frames:
    return _Frames(frames.ctypes.data, d["bits"], d["height"], d["width"], d.get("x0", 0),
                   d.get("y0", 0), d["row_stride"], d["frame_stride_bytes"], d.get("bit_order", 0))


def _as_frames(frames) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(frames, dtype=np.uint8))
    return a


def unpack(frames, d: dict, n: int) -> np.ndarray:
    """Pixel values [M, n] (pixel-major) of region ``d`` in the first n frames."""
    fr = _as_frames(frames)
    out = np.empty((d["height"] * d["width"], n), dtype=np.uint8)
    rc = lib().oracle_unpack(ctypes.byref(_desc(fr, d)), n, out.ctypes.data)
    if rc:
        raise ValueError(f"oracle_unpack failed ({rc})")
    return out


def correlate(frames_a, da: dict, frames_b, db: dict, n: int, rows=None, gamma=True):
    """Eq. (1) with exact integer sums. Returns dict(s_ab, s_a, s_b, gamma).

    rows=(r0, r1) computes only those rows of s_ab / gamma (others are left 0)."""
    fa, fb = _as_frames(frames_a), _as_frames(frames_b)
    Ma, Mb = da["height"] * da["width"], db["height"] * db["width"]
    s_ab = np.zeros((Ma, Mb), dtype=np.int64)
    s_a = np.zeros(Ma, dtype=np.int64)
    s_b = np.zeros(Mb, dtype=np.int64)
    g = np.zeros((Ma, Mb), dtype=np.float64) if gamma else None
    r0, r1 = rows if rows is not None else (0, 0)
    A, B = _desc(fa, da), _desc(fb, db)
    rc = lib().oracle_correlate(ctypes.byref(A), ctypes.byref(B), n, r0, r1, s_ab.ctypes.data,
                                s_a.ctypes.data, s_b.ctypes.data,
                                g.ctypes.data if g is not None else None)
    if rc:
        raise ValueError(f"oracle_correlate failed ({rc})")
    return {"s_ab": s_ab, "s_a": s_a, "s_b": s_b, "gamma": g}


def correlate_rows(frames_a, da: dict, frames_b, db: dict, n: int, r0: int, r1: int):
    """Rows r0 .. r1 - 1 of Eq. (1) only, for outputs too large to hold whole:
    returns dict(s_ab [r1 - r0][Mb], s_a, s_b, gamma [r1 - r0][Mb]).  The C routine
    indexes its outputs by the full row number and writes only rows r0 .. r1 - 1,
    so it is given addresses that place row r0 at the start of the row buffers."""
    fa, fb = _as_frames(frames_a), _as_frames(frames_b)
    Ma, Mb = da["height"] * da["width"], db["height"] * db["width"]
    assert 0 <= r0 < r1 <= Ma
    s_ab = np.zeros((r1 - r0, Mb), dtype=np.int64)
    g = np.zeros((r1 - r0, Mb), dtype=np.float64)
    s_a = np.zeros(Ma, dtype=np.int64)
    s_b = np.zeros(Mb, dtype=np.int64)
    shift = r0 * Mb * 8
    A, B = _desc(fa, da), _desc(fb, db)
    rc = lib().oracle_correlate(ctypes.byref(A), ctypes.byref(B), n, r0, r1,
                                ctypes.c_void_p(s_ab.ctypes.data - shift), s_a.ctypes.data, s_b.ctypes.data,
                                ctypes.c_void_p(g.ctypes.data - shift))
    if rc:
        raise ValueError(f"oracle_correlate failed ({rc})")
    return {"s_ab": s_ab, "s_a": s_a, "s_b": s_b, "gamma": g}


def refocus(gamma: np.ndarray, ha: int, wa: int, hb: int, wb: int, alpha, beta) -> np.ndarray:
    """Refocused stack [P, ha, wa] (float64) from Gamma [ha*wa, hb*wb] (float64)."""
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    assert g.shape == (ha * wa, hb * wb)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    be = np.ascontiguousarray(beta, dtype=np.float64)
    P = len(al)
    out = np.empty((P, ha, wa), dtype=np.float64)
    rc = lib().oracle_refocus(g.ctypes.data, ha, wa, hb, wb, al.ctypes.data, be.ctypes.data, P,
                              out.ctypes.data)
    if rc:
        raise ValueError(f"oracle_refocus failed ({rc})")
    return out


def refocus4d(gamma: np.ndarray, ha: int, wa: int, hb: int, wb: int, alpha, beta, gam, delta) -> np.ndarray:
    """4-D multilinear refocused stack [P, ha, wa] (float64) from Gamma [ha*wa, hb*wb]."""
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    assert g.shape == (ha * wa, hb * wb)
    co = [np.ascontiguousarray(v, dtype=np.float64) for v in (alpha, beta, gam, delta)]
    P = len(co[0])
    assert all(len(v) == P for v in co)
    out = np.empty((P, ha, wa), dtype=np.float64)
    rc = lib().oracle_refocus4d(g.ctypes.data, ha, wa, hb, wb, *[v.ctypes.data for v in co], P, out.ctypes.data)
    if rc:
        raise ValueError(f"oracle_refocus4d failed ({rc})")
    return out


def timed(fn, *args, **kw):
    t0 = time.perf_counter()
    r = fn(*args, **kw)
    return r, time.perf_counter() - t0
