"""Seeded synthetic camera frames for the five workload configurations.

Input bytes only: this module holds none of the method's arithmetic.  Both the
CUDA path's tests/benchmark and the CPU oracle consume what it makes.  The
scene recipe is documented at the top of ``gen.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

N_LEARN = 30
RUN_FRAMES = {1: 60, 2: 300, 3: 600, 4: 120}


def build(force: bool = False) -> str:
    """Compile gen.c (gcc -O2, OpenMP when available, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_num_streams.restype = ctypes.c_int
            lib.synth_num_streams.argtypes = [ctypes.c_int]
            lib.synth_shape.restype = ctypes.c_int
            lib.synth_shape.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_frame.restype = ctypes.c_int
            lib.synth_frame.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p]
            lib.synth_truth.restype = ctypes.c_int
            lib.synth_truth.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_brightness.restype = ctypes.c_double
            lib.synth_brightness.argtypes = [ctypes.c_int] * 3
            _lib = lib
        return _lib


def num_streams(cfg: int) -> int:
    n = _load().synth_num_streams(cfg)
    if n <= 0:
        raise ValueError(f"unknown configuration {cfg}")
    return n


def shape(cfg: int, stream: int = 0) -> tuple[int, int]:
    """(W, H) of a stream."""
    w, h = ctypes.c_int(), ctypes.c_int()
    if _load().synth_shape(cfg, stream, ctypes.byref(w), ctypes.byref(h)):
        raise ValueError(f"no stream {stream} in configuration {cfg}")
    return w.value, h.value


def _frame_into(cfg, stream, t, learn, out):
    if _load().synth_frame(cfg, stream, t, int(learn), out.ctypes.data):
        raise ValueError("bad synth_frame arguments")


def learn_frames(cfg: int, stream: int = 0, n: int = N_LEARN) -> np.ndarray:
    """(n, H, W, 3) uint8 user-free frames."""
    w, h = shape(cfg, stream)
    out = np.empty((n, h, w, 3), np.uint8)
    for i in range(n):
        _frame_into(cfg, stream, i, True, out[i])
    return out


def run_frame(cfg: int, stream: int, t: int, out: np.ndarray | None = None) -> np.ndarray:
    """Run frame t, (H, W, 3) uint8."""
    w, h = shape(cfg, stream)
    if out is None:
        out = np.empty((h, w, 3), np.uint8)
    assert out.shape == (h, w, 3) and out.dtype == np.uint8 and out.flags["C_CONTIGUOUS"]
    _frame_into(cfg, stream, t, False, out)
    return out


def run_frames(cfg: int, stream: int, t0: int, count: int) -> np.ndarray:
    w, h = shape(cfg, stream)
    out = np.empty((count, h, w, 3), np.uint8)
    for i in range(count):
        _frame_into(cfg, stream, t0 + i, False, out[i])
    return out


def truth(cfg: int, stream: int, t: int):
    """Ground truth of run frame t: (list of (cx, cy, a, b) ellipses, hand open)."""
    buf = np.zeros(8, np.float64)
    op = ctypes.c_int()
    n = _load().synth_truth(cfg, stream, t, buf.ctypes.data, ctypes.byref(op))
    if n < 0:
        raise ValueError("bad synth_truth arguments")
    return [tuple(buf[4 * k:4 * k + 4]) for k in range(n)], bool(op.value)


def brightness(cfg: int, stream: int, t: int) -> float:
    return _load().synth_brightness(cfg, stream, t)
