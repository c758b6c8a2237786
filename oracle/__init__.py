"""CPU oracle of the per-frame hand-isolation path (arXiv 1907.04393).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this package.  The product
path (``paper_1907_04393_gb300``) never imports it and shares no code with it.

This module is a thin ctypes wrapper around ``hmi_oracle.c`` (plain C, single
threaded), which it compiles with gcc on first use.  Every function below maps
one-to-one onto a C function whose comment cites the passage of the paper it
follows (Sec. 2 workflow, Sec. 3.1 mask building, Sec. 3.2 luminosity).

Parity status: every stage is pinned by ``tests/test_oracle_pins.py`` against
closed forms, library routines (scipy.ndimage, colorsys) and brute force.  The
readings of the paper's garbled or silent passages are pinned only against
themselves ("parity unpinned" against the authors' system, whose code,
thresholds and data are not available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hmi_oracle.c into liboracle.so (gcc, -O2, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Pointer(ctypes.Structure):
    _fields_ = [("valid", ctypes.c_int32), ("click", ctypes.c_int32),
                ("x", ctypes.c_float), ("y", ctypes.c_float),
                ("area", ctypes.c_uint32),
                ("x0", ctypes.c_int32), ("y0", ctypes.c_int32),
                ("x1", ctypes.c_int32), ("y1", ctypes.c_int32),
                ("label", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_u8p = _P
_I, _U32, _U64, _I64, _SZ = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_size_t


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "orc_learn_stats": (None, [_P, _I, _I, _I, _P, _P, _P, _P]),
            "orc_learn_meanstd": (None, [_P, _P, _I, _SZ, _P, _P]),
            "orc_band_low": (_I64, [_U32, _U32, _I, _I, _I]),
            "orc_band_high": (_I64, [_U32, _U32, _I, _I, _I]),
            "orc_learn_band": (None, [_P, _P, _P, _P, _I, _SZ, _I, _I, _I, _P, _P]),
            "orc_luma_sum": (_U64, [_P, _SZ]),
            "orc_ref_luma": (_U64, [_P, _I, _SZ]),
            "orc_gain": (_U32, [_U64, _U64, _U32, _U32]),
            "orc_apply_gain": (None, [_P, _SZ, _U32, _P]),
            "orc_hue": (_I, [_I, _I, _I]),
            "orc_hue_map": (None, [_P, _SZ, _P]),
            "orc_fg": (None, [_P, _P, _P, _SZ, _I, _I, _I, _P, _P, _P, _P]),
            "orc_erode": (None, [_P, _I, _I, _P]),
            "orc_dilate": (None, [_P, _I, _I, _P]),
            "orc_morph": (None, [_P, _I, _I, _I, _I, _P]),
            "orc_label": (_I, [_P, _I, _I, _P]),
            "orc_pointer_from_labels": (None, [_P, _I, _I, _U32, _P]),
            "orc_click_update": (None, [_P, _P, _P, _I, _I, _I, _P]),
            "orc_relearn_reset": (None, [_SZ, _P, _P, _P, _P, _P]),
            "orc_relearn_accumulate": (None, [_P, _P, _P, _SZ, _P, _P, _P, _P, _P]),
            "orc_relearn_apply": (None, [_P, _P, _P, _P, _P, _SZ, _I, _I, _I, _I, _P, _P]),
            "orc_relearn_in_window": (_I, [ctypes.c_longlong, _I, _I]),
            "orc_pointer_select": (None, [_P, _I, _I, _U32, _I, _P, _P]),
            "orc_diamond_angle": (ctypes.c_int32, [_I64, _I64]),
            "orc_interface_event": (None, [_I, ctypes.c_int32, ctypes.c_int32, _I, _P, _I, _P, _P]),
            "orc_process_frame": (None, [_P, _I, _I, _P, _P, _U64, _I, _I, _I, _I, _I,
                                         _U32, _U32, _U32, _I, _I, _I, _I, _P, _P, _P, _P,
                                         _P, _P, _P, _P]),
            "orc_process_frame_bg": (None, [_P, _I, _I, _P, _P, _P, _U64, _I, _I, _I, _I, _I,
                                            _U32, _U32, _U32, _I, _I, _I, _I, _P, _P, _P, _P,
                                            _P, _P, _P, _P]),
            "orc_mixture_step": (None, [_P, _P, _P, _P, _SZ, _I, _P, _U32, _I, _I, _I, _I,
                                        _U32, _U32, _P]),
            "orc_mixture_learn": (None, [_P, _I, _SZ, _I, _P, _P, _P, _P, _I, _I, _I, _U32,
                                         _U32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


# --------------------------------------------------------------------------- #
# Default parameters (the same documented defaults as the library's).        #
# --------------------------------------------------------------------------- #
DEFAULTS = dict(gray_tol=15, hue_lo=1472, hue_hi=256, bg_margin=2, bg_k_num=5,
                bg_k_den=2, open_iters=1, close_iters=1, gain_min_q16=32768,
                gain_max_q16=131072, min_area=50, click_on_pct=80,
                click_off_pct=90, click_window=30,
                relearn_frames=0, relearn_min=0, relearn_period=0, track_max_dist=0,
                bg_model=0, mix_k=3, mix_bg_pct=70, mix_sigma0=15, mix_sigma_min=2,
                mix_rate_n=256)


def params(**over) -> dict:
    p = dict(DEFAULTS)
    unknown = set(over) - set(p)
    if unknown:
        raise KeyError(f"unknown oracle params {sorted(unknown)}")
    p.update(over)
    return p


# --------------------------------------------------------------------------- #
# Stage functions                                                            #
# --------------------------------------------------------------------------- #
def learn_stats(frames: np.ndarray):
    """frames: (n, H, W, 3) uint8 -> (S, Q, vmin, vmax) shaped (H, W, 3)."""
    frames = _u8(frames)
    n, h, w, _ = frames.shape
    S = np.empty((h, w, 3), np.uint32)
    Q = np.empty((h, w, 3), np.uint32)
    vmin = np.empty((h, w, 3), np.uint8)
    vmax = np.empty((h, w, 3), np.uint8)
    _load().orc_learn_stats(_ptr(frames), n, w, h, _ptr(S), _ptr(Q), _ptr(vmin), _ptr(vmax))
    return S, Q, vmin, vmax


def learn_meanstd(S: np.ndarray, Q: np.ndarray, n: int):
    S = np.ascontiguousarray(S, np.uint32)
    Q = np.ascontiguousarray(Q, np.uint32)
    mean = np.empty(S.shape, np.float32)
    std = np.empty(S.shape, np.float32)
    _load().orc_learn_meanstd(_ptr(S), _ptr(Q), n, S.size, _ptr(mean), _ptr(std))
    return mean, std


def band_low(S: int, Q: int, n: int, kn: int, kd: int) -> int:
    if kd < 1:
        raise ValueError("kd must be >= 1")
    return _load().orc_band_low(S, Q, n, kn, kd)


def band_high(S: int, Q: int, n: int, kn: int, kd: int) -> int:
    if kd < 1:
        raise ValueError("kd must be >= 1")
    return _load().orc_band_high(S, Q, n, kn, kd)


def learn_band(S, Q, vmin, vmax, n, kn, kd, delta):
    if kd < 1:
        raise ValueError("kd must be >= 1")
    S = np.ascontiguousarray(S, np.uint32)
    Q = np.ascontiguousarray(Q, np.uint32)
    vmin, vmax = _u8(vmin), _u8(vmax)
    lo = np.empty(S.shape, np.uint8)
    hi = np.empty(S.shape, np.uint8)
    _load().orc_learn_band(_ptr(S), _ptr(Q), _ptr(vmin), _ptr(vmax), n, S.size, kn, kd,
                           delta, _ptr(lo), _ptr(hi))
    return lo, hi


def luma_sum(frame: np.ndarray) -> int:
    frame = _u8(frame)
    return _load().orc_luma_sum(_ptr(frame), frame.size // 3)


def ref_luma(frames: np.ndarray) -> int:
    frames = _u8(frames)
    n = frames.shape[0]
    return _load().orc_ref_luma(_ptr(frames), n, frames[0].size // 3)


def gain(sy: int, syref: int, gmin: int, gmax: int) -> int:
    return _load().orc_gain(sy, syref, gmin, gmax)


def apply_gain(frame: np.ndarray, g: int) -> np.ndarray:
    frame = _u8(frame)
    out = np.empty_like(frame)
    _load().orc_apply_gain(_ptr(frame), frame.size, g, _ptr(out))
    return out


def hue(r: int, g: int, b: int) -> int:
    return _load().orc_hue(int(r), int(g), int(b))


def hue_map(c: np.ndarray) -> np.ndarray:
    """Integer hue of every pixel of (..., 3) uint8, int16, -1 where undefined."""
    c = _u8(c)
    out = np.empty(c.shape[:-1], np.int16)
    _load().orc_hue_map(_ptr(c), c.size // 3, _ptr(out))
    return out


def fg(c: np.ndarray, lo: np.ndarray, hi: np.ndarray, gray_tol: int, hue_lo: int, hue_hi: int):
    """Gain-corrected frame (..., 3) -> (fg1, fg2, fg3, raw) shaped like c[..., 0]."""
    c, lo, hi = _u8(c), _u8(lo), _u8(hi)
    assert c.shape == lo.shape == hi.shape and c.shape[-1] == 3
    shp = c.shape[:-1]
    outs = [np.empty(shp, np.uint8) for _ in range(4)]
    _load().orc_fg(_ptr(c), _ptr(lo), _ptr(hi), c.size // 3, gray_tol, hue_lo, hue_hi,
                   *[_ptr(o) for o in outs])
    return tuple(outs)


def erode(m: np.ndarray) -> np.ndarray:
    m = _u8(m)
    out = np.empty_like(m)
    h, w = m.shape
    _load().orc_erode(_ptr(m), w, h, _ptr(out))
    return out


def dilate(m: np.ndarray) -> np.ndarray:
    m = _u8(m)
    out = np.empty_like(m)
    h, w = m.shape
    _load().orc_dilate(_ptr(m), w, h, _ptr(out))
    return out


def morph(m: np.ndarray, open_iters: int, close_iters: int) -> np.ndarray:
    m = _u8(m)
    out = np.empty_like(m)
    h, w = m.shape
    _load().orc_morph(_ptr(m), w, h, open_iters, close_iters, _ptr(out))
    return out


def label(m: np.ndarray):
    """Binary mask (H, W) -> (labels int32 (H, W), component count)."""
    m = _u8(m)
    h, w = m.shape
    lab = np.empty((h, w), np.int32)
    n = _load().orc_label(_ptr(m), w, h, _ptr(lab))
    return lab, n


def pointer_select(labels: np.ndarray, min_area: int, max_dist: int, track=None):
    """Tracked pointer choice; returns (pointer dict, new track (valid, x, y))."""
    labels = np.ascontiguousarray(labels, np.int32)
    h, w = labels.shape
    tr = np.zeros(3, np.int32) if track is None else np.array(track, np.int32)
    p = Pointer()
    _load().orc_pointer_select(_ptr(labels), w, h, min_area, max_dist, _ptr(tr), ctypes.byref(p))
    return p.as_dict(), tuple(int(v) for v in tr)


def diamond_angle(dx: int, dy: int) -> int:
    return _load().orc_diamond_angle(int(dx), int(dy))


EVENT_FIELDS = ("zone", "event", "on_wheel", "steer", "left", "right", "throttle")


def interface_event(valid: bool, px: int, py: int, click: int, zones, wheel) -> dict:
    """zones: [(x0, y0, x1, y1, event)], wheel: (on, cx, cy, r_in, r_out, dead_zone)."""
    z = np.ascontiguousarray(np.array(zones, np.int32).reshape(-1, 5)) if len(zones) else np.zeros((1, 5), np.int32)
    wl = np.ascontiguousarray(np.array(wheel, np.int32))
    out = np.zeros(7, np.int32)
    _load().orc_interface_event(int(valid), int(px), int(py), int(click), _ptr(z), len(zones), _ptr(wl), _ptr(out))
    return dict(zip(EVENT_FIELDS, (int(v) for v in out)))


def pointer_from_labels(labels: np.ndarray, min_area: int) -> dict:
    labels = np.ascontiguousarray(labels, np.int32)
    h, w = labels.shape
    p = Pointer()
    _load().orc_pointer_from_labels(_ptr(labels), w, h, min_area, ctypes.byref(p))
    return p.as_dict()


class ClickState:
    """Per-stream click state machine (history of the last `window` valid areas)."""

    def __init__(self, window: int):
        self.window = int(window)
        self.click = ctypes.c_int32(0)
        self.count = ctypes.c_int32(0)
        self.hist = np.zeros(max(self.window, 1), np.uint32)

    def update(self, ptr: dict, on_pct: int, off_pct: int) -> dict:
        p = Pointer(**{k: ptr[k] for k, _ in Pointer._fields_})
        _load().orc_click_update(ctypes.byref(self.click), _ptr(self.hist),
                                 ctypes.byref(self.count), self.window, on_pct, off_pct,
                                 ctypes.byref(p))
        return p.as_dict()


class Relearn:
    """Re-learning sums of one stream (orc_relearn_*), shaped (H, W, 3) / (H, W)."""

    def __init__(self, h: int, w: int):
        self.S = np.empty((h, w, 3), np.uint32)
        self.Q = np.empty((h, w, 3), np.uint32)
        self.vmin = np.empty((h, w, 3), np.uint8)
        self.vmax = np.empty((h, w, 3), np.uint8)
        self.cnt = np.empty((h, w), np.uint8)
        _load().orc_relearn_reset(h * w, _ptr(self.S), _ptr(self.Q), _ptr(self.vmin),
                                  _ptr(self.vmax), _ptr(self.cnt))

    def accumulate(self, c, lo, hi) -> None:
        _load().orc_relearn_accumulate(_ptr(c), _ptr(lo), _ptr(hi), self.cnt.size, _ptr(self.S),
                                       _ptr(self.Q), _ptr(self.vmin), _ptr(self.vmax),
                                       _ptr(self.cnt))

    def apply(self, min_cnt: int, kn: int, kd: int, delta: int, lo, hi) -> None:
        _load().orc_relearn_apply(_ptr(self.S), _ptr(self.Q), _ptr(self.vmin), _ptr(self.vmax),
                                  _ptr(self.cnt), self.cnt.size, min_cnt, kn, kd, delta,
                                  _ptr(lo), _ptr(hi))


def relearn_in_window(f: int, period: int, frames: int) -> bool:
    return bool(_load().orc_relearn_in_window(f, period, frames))


class _OrcMixture(ctypes.Structure):
    _fields_ = [("W", ctypes.c_void_p), ("M", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("K", ctypes.c_int), ("t", ctypes.c_uint32),
                ("rate_n", ctypes.c_int), ("bg_pct", ctypes.c_int), ("ln", ctypes.c_int),
                ("ld", ctypes.c_int), ("v_init", ctypes.c_uint32), ("v_min", ctypes.c_uint32)]


class Mixture:
    """Per-pixel Gaussian mixture of one stream (orc_mixture_step, Sec. 2 / Sec. 3.3).

    Planes: W (K, npx) Q15 weights, M (K, 3, npx) Q8 means, V (K, npx) Q4
    variances, C (K, npx) match counts, in storage (fitness) order; t is the
    number of frames seen so far."""

    def __init__(self, npx: int, K: int, rate_n: int, bg_pct: int, ln: int, ld: int,
                 sigma0: int, sigma_min: int):
        self.npx, self.K = int(npx), int(K)
        self.rate_n, self.bg_pct, self.ln, self.ld = int(rate_n), int(bg_pct), int(ln), int(ld)
        self.v_init, self.v_min = 16 * int(sigma0) ** 2, 16 * int(sigma_min) ** 2
        self.W = np.zeros((K, npx), np.uint16)
        self.M = np.zeros((K, 3, npx), np.uint16)
        self.V = np.zeros((K, npx), np.uint16)
        self.C = np.zeros((K, npx), np.uint16)
        self.t = 0

    @classmethod
    def from_params(cls, npx: int, p: dict) -> "Mixture":
        return cls(npx, p["mix_k"], p["mix_rate_n"], p["mix_bg_pct"], p["bg_k_num"],
                   p["bg_k_den"], p["mix_sigma0"], p["mix_sigma_min"])

    def step(self, x: np.ndarray, classify: bool = True):
        """One frame x (npx x 3 bytes, or any shape of npx*3 bytes).  Returns
        fg1 (npx uint8) when classify, else None."""
        x = _u8(x).reshape(-1)
        assert x.size == 3 * self.npx
        self.t += 1
        fg1 = np.empty(self.npx, np.uint8) if classify else None
        _load().orc_mixture_step(_ptr(self.W), _ptr(self.M), _ptr(self.V), _ptr(self.C), self.npx,
                                 self.K, _ptr(x), self.t, self.rate_n, self.bg_pct, self.ln, self.ld,
                                 self.v_init, self.v_min, _ptr(fg1))
        return fg1

    def learn(self, frames: np.ndarray) -> None:
        """The learning frames in order from an empty model (orc_mixture_learn)."""
        frames = _u8(frames)
        n = frames.shape[0]
        assert frames[0].size == 3 * self.npx
        _load().orc_mixture_learn(_ptr(frames), n, self.npx, self.K, _ptr(self.W), _ptr(self.M),
                                  _ptr(self.V), _ptr(self.C), self.rate_n, self.ln, self.ld,
                                  self.v_init, self.v_min)
        self.t = n

    def descriptor(self, t: int) -> _OrcMixture:
        return _OrcMixture(_ptr(self.W), _ptr(self.M), _ptr(self.V), _ptr(self.C), self.K, t,
                           self.rate_n, self.bg_pct, self.ln, self.ld, self.v_init, self.v_min)

    def planes(self) -> np.ndarray:
        """All state as (6K, npx) uint16: W[k], M[k][ch], V[k], C[k]."""
        return np.concatenate([self.W, self.M.reshape(3 * self.K, -1), self.V, self.C])


class OracleStream:
    """The whole path for one camera stream: learn once, then process frames."""

    def __init__(self, w: int, h: int, **over):
        self.w, self.h = int(w), int(h)
        self.p = params(**over)
        self.learned = False
        self.click = ClickState(self.p["click_window"])

    def learn(self, frames: np.ndarray) -> None:
        frames = _u8(frames)
        assert frames.shape[1:] == (self.h, self.w, 3)
        n = frames.shape[0]
        S, Q, vmin, vmax = learn_stats(frames)
        self.n = n
        self.S, self.Q, self.vmin, self.vmax = S, Q, vmin, vmax
        self.lo, self.hi = learn_band(S, Q, vmin, vmax, n, self.p["bg_k_num"],
                                      self.p["bg_k_den"], self.p["bg_margin"])
        self.syref = ref_luma(frames)
        self.mix = None
        if self.p["bg_model"] == 1:
            self.mix = Mixture.from_params(self.h * self.w, self.p)
            self.mix.learn(frames)
        self.learned = True
        self._reset_relearn()

    def set_interface(self, zones, wheel) -> None:
        """Headless Interface module and wheel (orc_interface_event)."""
        self.ui = (list(zones), tuple(wheel))

    def _reset_relearn(self) -> None:
        self.frames = 0
        self.track = np.zeros(3, np.int32)   # (valid, x, y) of the tracked point
        self.relearn = Relearn(self.h, self.w) if self.p["relearn_frames"] > 0 else None

    def set_background(self, S, Q, vmin, vmax, n: int, syref: int) -> None:
        """Install learned sums directly (the state learning would leave)."""
        assert self.p["bg_model"] == 0, "a mixture stream learns from frames"
        self.mix = None
        self.n = int(n)
        self.S = np.ascontiguousarray(S, np.uint32)
        self.Q = np.ascontiguousarray(Q, np.uint32)
        self.vmin, self.vmax = _u8(vmin), _u8(vmax)
        self.lo, self.hi = learn_band(self.S, self.Q, self.vmin, self.vmax, self.n,
                                      self.p["bg_k_num"], self.p["bg_k_den"], self.p["bg_margin"])
        self.syref = int(syref)
        self.click = ClickState(self.p["click_window"])
        self.learned = True
        self._reset_relearn()

    def stats(self):
        return learn_meanstd(self.S, self.Q, self.n)

    def process(self, frame: np.ndarray, want_labels: bool = True):
        """Returns (mask uint8 (H,W), labels int32 (H,W) or None, pointer dict, gain)."""
        assert self.learned
        frame = _u8(frame)
        assert frame.shape == (self.h, self.w, 3)
        p = self.p
        mask = np.empty((self.h, self.w), np.uint8)
        labels = np.empty((self.h, self.w), np.int32) if want_labels else None
        ptr = Pointer()
        g = ctypes.c_uint32(0)
        c = self.click
        mix = getattr(self, "mix", None)
        desc = mix.descriptor(mix.t + 1) if mix is not None else None
        _load().orc_process_frame_bg(
            _ptr(frame), self.w, self.h, _ptr(self.lo), _ptr(self.hi),
            ctypes.byref(desc) if desc is not None else None, self.syref,
            p["gray_tol"], p["hue_lo"], p["hue_hi"], p["open_iters"], p["close_iters"],
            p["gain_min_q16"], p["gain_max_q16"], p["min_area"], p["click_on_pct"],
            p["click_off_pct"], c.window, p["track_max_dist"], _ptr(self.track),
            ctypes.byref(c.click), _ptr(c.hist),
            ctypes.byref(c.count), _ptr(mask), _ptr(labels), ctypes.byref(ptr),
            ctypes.byref(g))
        if mix is not None:
            mix.t += 1
        # the Interface module's event from this frame's pointer (Sec. 2, 4)
        if getattr(self, "ui", None) is not None:
            pd = ptr.as_dict()
            self.event = interface_event(pd["valid"], self.track[1], self.track[2], pd["click"],
                                         self.ui[0], self.ui[1])
        # re-learning (Sec. 3.3), after this frame's classification
        self.frames += 1
        if self.relearn is not None and relearn_in_window(self.frames, p["relearn_period"],
                                                           p["relearn_frames"]):
            self.relearn.accumulate(apply_gain(frame, g.value), self.lo, self.hi)
            if self.frames % p["relearn_period"] == 0:
                self.relearn.apply(p["relearn_min"], p["bg_k_num"], p["bg_k_den"], p["bg_margin"],
                                   self.lo, self.hi)
        return mask, labels, ptr.as_dict(), g.value
