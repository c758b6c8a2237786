"""Python binding of libhmi.so: the C ABI of include/hmi.h, same names.

Argument marshalling only.  Every step of the path runs in the library's CUDA
kernels; this module has no compute of its own and no fallback: if the
library is missing or cannot be loaded, importing the binding raises.

Buffers are passed as raw addresses.  ``_addr`` accepts a numpy array (host
memory), a torch tensor (host or CUDA memory, via ``data_ptr``) or an int.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HMI_OK = 0
HMI_ERR_INVALID_ARG = -1
HMI_ERR_NOT_LEARNED = -2
HMI_ERR_NO_MEMORY = -3
HMI_ERR_DEVICE = -4
HMI_ERR_DEVICE_TIMEOUT = -5
HMI_LEARNING = 1          # server results only: a background-learning frame
HMI_TICK_KERNELS = 9


class hmi_params(ctypes.Structure):
    _fields_ = [("gain_min_q16", ctypes.c_uint32), ("gain_max_q16", ctypes.c_uint32),
                ("min_area", ctypes.c_uint32), ("hue_lo", ctypes.c_uint16),
                ("hue_hi", ctypes.c_uint16), ("click_window", ctypes.c_uint16),
                ("gray_tol", ctypes.c_uint8), ("bg_margin", ctypes.c_uint8),
                ("bg_k_num", ctypes.c_uint8), ("bg_k_den", ctypes.c_uint8),
                ("open_iters", ctypes.c_uint8), ("close_iters", ctypes.c_uint8),
                ("click_on_pct", ctypes.c_uint8), ("click_off_pct", ctypes.c_uint8),
                ("relearn_frames", ctypes.c_uint8), ("relearn_min", ctypes.c_uint8),
                ("relearn_period", ctypes.c_uint16), ("track_max_dist", ctypes.c_uint16),
                ("bg_model", ctypes.c_uint8), ("mix_k", ctypes.c_uint8),
                ("mix_bg_pct", ctypes.c_uint8), ("mix_sigma0", ctypes.c_uint8),
                ("mix_sigma_min", ctypes.c_uint8), ("mix_pad", ctypes.c_uint8),
                ("mix_rate_n", ctypes.c_uint16)]


class hmi_pointer(ctypes.Structure):
    _fields_ = [("valid", ctypes.c_int32), ("click", ctypes.c_int32),
                ("x", ctypes.c_float), ("y", ctypes.c_float), ("area", ctypes.c_uint32),
                ("x0", ctypes.c_int32), ("y0", ctypes.c_int32),
                ("x1", ctypes.c_int32), ("y1", ctypes.c_int32), ("label", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class hmi_server_result(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int32), ("status", ctypes.c_int32), ("tag", ctypes.c_uint64),
                ("submit_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64),
                ("pointer", hmi_pointer)]


HMI_MAX_ZONES = 16


class hmi_zone(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("x1", ctypes.c_int32),
                ("y1", ctypes.c_int32), ("event", ctypes.c_int32)]


class hmi_interface(ctypes.Structure):
    _fields_ = [("nzones", ctypes.c_int32), ("zones", hmi_zone * HMI_MAX_ZONES),
                ("wheel_on", ctypes.c_int32), ("wheel_cx", ctypes.c_int32), ("wheel_cy", ctypes.c_int32),
                ("wheel_r_in", ctypes.c_int32), ("wheel_r_out", ctypes.c_int32),
                ("dead_zone", ctypes.c_int32)]


class hmi_event(ctypes.Structure):
    _fields_ = [("zone", ctypes.c_int32), ("event", ctypes.c_int32), ("on_wheel", ctypes.c_int32),
                ("steer", ctypes.c_int32), ("left", ctypes.c_int32), ("right", ctypes.c_int32),
                ("throttle", ctypes.c_int32), ("frame", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class hmi_tuning(ctypes.Structure):
    _fields_ = [("piece_chunks", ctypes.c_int32), ("luma_ctas_per_sm", ctypes.c_int32),
                ("skin_ctas_per_sm", ctypes.c_int32), ("cc_ctas_per_sm", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("pipeline_depth", ctypes.c_int32),
                ("fused", ctypes.c_int32), ("queue_lag", ctypes.c_int32),
                ("merge_threads", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class hmi_server_round(ctypes.Structure):
    _fields_ = [("start_ns", ctypes.c_uint64), ("setup_ns", ctypes.c_uint64),
                ("issued_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64),
                ("frames", ctypes.c_int32), ("learning", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("replanned", ctypes.c_int32),
                ("created", ctypes.c_int32), ("retired", ctypes.c_int32)]


POINTER_DTYPE = np.dtype([(k, np.dtype(t._type_)) for k, t in hmi_pointer._fields_])
assert POINTER_DTYPE.itemsize == ctypes.sizeof(hmi_pointer) == 40

_P = ctypes.c_void_p
_I = ctypes.c_int

# name -> (restype, argtypes), one entry per function of include/hmi.h
SIGNATURES = {
    "hmi_default_params": (_I, [ctypes.POINTER(hmi_params)]),
    "hmi_create_stream": (_P, [_I, _I, ctypes.POINTER(hmi_params)]),
    "hmi_destroy_stream": (None, [_P]),
    "hmi_learn_background": (_I, [_P, _P, _I]),
    "hmi_process_frame": (_I, [_P, _P, _P, _P]),
    "hmi_process_frame_async": (_I, [_P, _P, _P, _P, _P]),
    "hmi_process_batch": (_I, [_P, _I, _P, _P, _P]),
    "hmi_batch_create": (_P, [_P, _I]),
    "hmi_batch_destroy": (None, [_P]),
    "hmi_batch_process": (_I, [_P, _P, _P, _P]),
    "hmi_batch_process_async": (_I, [_P, _P, _P, _P, _P, _I]),
    "hmi_batch_set_groups": (_I, [_P, _I]),
    "hmi_batch_set_loop_limit": (_I, [_P, ctypes.c_uint32]),
    "hmi_batch_get_groups": (_I, [_P]),
    "hmi_batch_set_tuning": (_I, [_P, ctypes.POINTER(hmi_tuning)]),
    "hmi_batch_get_tuning": (_I, [_P, ctypes.POINTER(hmi_tuning)]),
    "hmi_batch_autotune": (_I, [_P, _P, _I, _I, ctypes.POINTER(hmi_tuning), ctypes.POINTER(ctypes.c_double)]),
    "hmi_batch_process_pipelined": (_I, [_P, _P, _P, _P, _P, _I]),
    "hmi_batch_flush": (_I, [_P, _P]),
    "hmi_batch_profile": (_I, [_P, _I]),
    "hmi_batch_profile_read": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
    "hmi_batch_profile_kernels": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double), _I]),
    "hmi_get_background_stats": (_I, [_P, _P, _P]),
    "hmi_get_labels": (_I, [_P, _P]),
    "hmi_get_band": (_I, [_P, _P, _P]),
    "hmi_get_mixture": (_I, [_P, _P]),
    "hmi_set_interface": (_I, [_P, ctypes.POINTER(hmi_interface)]),
    "hmi_get_event": (_I, [_P, ctypes.POINTER(hmi_event)]),
    "hmi_export_background": (_I, [_P, _P, _P, _P, _P, _P, _P,
                                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_I)]),
    "hmi_import_background": (_I, [_P, _P, _P, _P, _P, _I, ctypes.c_uint64]),
    "hmi_get_last_gain": (_I, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "hmi_stream_device_bytes": (ctypes.c_size_t, [_I, _I, ctypes.POINTER(hmi_params)]),
    "hmi_frame_gain_noalloc": (_I, [_P, _I, _I, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    _P, _P]),
    "hmi_server_create": (_P, [ctypes.c_size_t, _I]),
    "hmi_server_destroy": (None, [_P]),
    "hmi_server_admit": (_I, [_P, _I, _I, ctypes.POINTER(hmi_params), _P, _I, ctypes.POINTER(_I)]),
    "hmi_server_release": (_I, [_P, _I]),
    "hmi_server_submit": (_I, [_P, _I, _P, ctypes.c_uint64]),
    "hmi_server_submit_ref": (_I, [_P, _I, _P, ctypes.c_uint64]),
    "hmi_server_poll": (_I, [_P, ctypes.POINTER(hmi_server_result), _I, _I]),
    "hmi_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_uint64),
                              ctypes.POINTER(ctypes.c_uint64)]),
    "hmi_server_now_ns": (ctypes.c_uint64, []),
    "hmi_server_rounds": (_I, [_P, ctypes.POINTER(hmi_server_round), _I]),
    "hmi_last_error": (_I, []),
    "hmi_status_string": (ctypes.c_char_p, [_I]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libhmi.so (building it first if it is missing or stale).  With
    HMI_DEBUG_BUILD=1 in the environment, the debug build (every computed index
    of the per-pixel kernels bounds-checked) is loaded instead."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("HMI_DEBUG_BUILD") == "1"
    path = _build.LIB_DEBUG if debug else _build.LIB
    if build_if_missing and not _build.up_to_date(debug):
        _build.build(debug=debug)
    if not os.path.exists(path):
        raise RuntimeError(f"libhmi.so not found at {path}; run the build first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class HmiError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = load().hmi_status_string(status).decode()
        super().__init__(f"{what}: {msg} ({status})")


def _check(status: int, what: str) -> int:
    if status != HMI_OK:
        raise HmiError(status, what)
    return status


def _addr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "buffers must be contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):          # torch.Tensor
        assert x.is_contiguous(), "buffers must be contiguous"
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _ptr_array(items) -> ctypes.Array:
    if isinstance(items, ctypes.Array):   # built once by ptr_array and reused
        return items
    arr = (ctypes.c_void_p * len(items))()
    for i, x in enumerate(items):
        arr[i] = _addr(x)
    return arr


def ptr_array(items) -> ctypes.Array:
    """The C array of buffer addresses that the batch calls take for their
    frames and masks.  Passing one built once (the buffers must stay alive and
    in place) saves converting every tensor on every call."""
    return _ptr_array(list(items))


# --------------------------------------------------------------------------- #
# Same-name wrappers of the C ABI                                             #
# --------------------------------------------------------------------------- #
def hmi_default_params(**over) -> hmi_params:
    p = hmi_params()
    _check(load().hmi_default_params(ctypes.byref(p)), "hmi_default_params")
    for k, v in over.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def hmi_create_stream(w: int, h: int, params: hmi_params | None = None) -> int:
    s = load().hmi_create_stream(w, h, ctypes.byref(params) if params is not None else None)
    if not s:
        raise HmiError(load().hmi_last_error(), "hmi_create_stream")
    return s


def hmi_destroy_stream(s: int) -> None:
    load().hmi_destroy_stream(s)


def hmi_learn_background(s: int, frames, n: int) -> None:
    _check(load().hmi_learn_background(s, _addr(frames), n), "hmi_learn_background")


def hmi_process_frame(s: int, frame, mask_out=None, pointer_out: hmi_pointer | None = None) -> None:
    _check(load().hmi_process_frame(s, _addr(frame), _addr(mask_out),
                                    ctypes.byref(pointer_out) if pointer_out is not None else None),
           "hmi_process_frame")


def hmi_process_frame_async(s: int, frame, mask_out, pointer_out, cuda_stream: int) -> None:
    _check(load().hmi_process_frame_async(s, _addr(frame), _addr(mask_out), _addr(pointer_out),
                                          cuda_stream), "hmi_process_frame_async")


def hmi_process_batch(streams, frames, masks=None, ptrs=None) -> None:
    n = len(streams)
    sa = (ctypes.c_void_p * n)(*streams)
    fa = _ptr_array(frames)
    ma = _ptr_array(masks) if masks is not None else None
    _check(load().hmi_process_batch(sa, n, fa, ma, _addr(ptrs)), "hmi_process_batch")


def hmi_batch_create(streams) -> int:
    n = len(streams)
    sa = (ctypes.c_void_p * n)(*streams)
    b = load().hmi_batch_create(sa, n)
    if not b:
        raise HmiError(load().hmi_last_error(), "hmi_batch_create")
    return b


def hmi_batch_destroy(b: int) -> None:
    load().hmi_batch_destroy(b)


def hmi_batch_process(b: int, frames, masks=None, ptrs=None) -> None:
    fa = _ptr_array(frames)
    ma = _ptr_array(masks) if masks is not None else None
    _check(load().hmi_batch_process(b, fa, ma, _addr(ptrs)), "hmi_batch_process")


def hmi_batch_process_async(b: int, frames, masks, ptrs, cuda_stream: int, use_graph: bool) -> None:
    fa = _ptr_array(frames)
    ma = _ptr_array(masks) if masks is not None else None
    _check(load().hmi_batch_process_async(b, fa, ma, _addr(ptrs), cuda_stream, int(use_graph)),
           "hmi_batch_process_async")


def hmi_batch_set_tuning(b: int, tuning) -> None:
    t = tuning if isinstance(tuning, hmi_tuning) else hmi_tuning(**tuning)
    _check(load().hmi_batch_set_tuning(b, ctypes.byref(t)), "hmi_batch_set_tuning")


def hmi_batch_get_tuning(b: int) -> dict:
    t = hmi_tuning()
    _check(load().hmi_batch_get_tuning(b, ctypes.byref(t)), "hmi_batch_get_tuning")
    return t.as_dict()


def hmi_batch_autotune(b: int, frames, ticks: int = 50, pipelined: bool = True) -> tuple[dict, float]:
    """Search and apply the batch's launch shape; (tuning, microseconds per tick)."""
    t, us = hmi_tuning(), ctypes.c_double()
    _check(load().hmi_batch_autotune(b, _ptr_array(frames), ticks, int(pipelined), ctypes.byref(t),
                                     ctypes.byref(us)), "hmi_batch_autotune")
    return t.as_dict(), us.value


def hmi_batch_process_pipelined(b: int, frames, masks, ptrs, cuda_stream: int, use_graph: bool) -> None:
    """Stage 1 of these frames beside stage 2 of the previous call's frames;
    this call's results are complete after the next call or hmi_batch_flush."""
    fa = _ptr_array(frames)
    ma = _ptr_array(masks) if masks is not None else None
    _check(load().hmi_batch_process_pipelined(b, fa, ma, _addr(ptrs), cuda_stream, int(use_graph)),
           "hmi_batch_process_pipelined")


def hmi_batch_flush(b: int, cuda_stream: int) -> None:
    _check(load().hmi_batch_flush(b, cuda_stream), "hmi_batch_flush")


def hmi_batch_set_loop_limit(b: int, limit: int) -> None:
    """Bound of the batch's device loops and waits (0: the default)."""
    _check(load().hmi_batch_set_loop_limit(b, limit), "hmi_batch_set_loop_limit")


def hmi_batch_set_groups(b: int, groups: int) -> None:
    _check(load().hmi_batch_set_groups(b, groups), "hmi_batch_set_groups")


def hmi_batch_get_groups(b: int) -> int:
    g = load().hmi_batch_get_groups(b)
    if g < 0:
        raise HmiError(g, "hmi_batch_get_groups")
    return g


def hmi_batch_profile(b: int, max_ticks: int) -> None:
    _check(load().hmi_batch_profile(b, max_ticks), "hmi_batch_profile")


TICK_KERNELS = ("luma", "classify", "mixture", "relearn", "relearn_band", "skin", "morphology",
                "block_components", "finish")


def hmi_batch_profile_kernels(b: int) -> tuple[int, dict]:
    """(ticks timed, {kernel name: summed milliseconds}) in tick order."""
    t = ctypes.c_int()
    ms = (ctypes.c_double * len(TICK_KERNELS))()
    _check(load().hmi_batch_profile_kernels(b, ctypes.byref(t), ms, len(TICK_KERNELS)),
           "hmi_batch_profile_kernels")
    return t.value, dict(zip(TICK_KERNELS, list(ms)))


def hmi_batch_profile_read(b: int) -> tuple[int, float]:
    t, ms = ctypes.c_int(), ctypes.c_double()
    _check(load().hmi_batch_profile_read(b, ctypes.byref(t), ctypes.byref(ms)), "hmi_batch_profile_read")
    return t.value, ms.value


def hmi_get_background_stats(s: int, mean, std) -> None:
    _check(load().hmi_get_background_stats(s, _addr(mean), _addr(std)), "hmi_get_background_stats")


def hmi_get_labels(s: int, labels) -> None:
    _check(load().hmi_get_labels(s, _addr(labels)), "hmi_get_labels")


def make_interface(zones=(), wheel=None) -> hmi_interface:
    """zones: [(x0, y0, x1, y1, event)], wheel: (cx, cy, r_in, r_out, dead_zone) or None."""
    ui = hmi_interface()
    ui.nzones = len(zones)
    for k, z in enumerate(zones):
        ui.zones[k] = hmi_zone(*z)
    if wheel is not None:
        ui.wheel_on = 1
        ui.wheel_cx, ui.wheel_cy, ui.wheel_r_in, ui.wheel_r_out, ui.dead_zone = wheel
    return ui


def hmi_set_interface(s: int, ui: hmi_interface) -> None:
    _check(load().hmi_set_interface(s, ctypes.byref(ui)), "hmi_set_interface")


def hmi_get_event(s: int) -> dict:
    e = hmi_event()
    _check(load().hmi_get_event(s, ctypes.byref(e)), "hmi_get_event")
    return e.as_dict()


def hmi_get_band(s: int, lo, hi) -> None:
    _check(load().hmi_get_band(s, _addr(lo), _addr(hi)), "hmi_get_band")


def hmi_get_mixture(s: int, out) -> None:
    _check(load().hmi_get_mixture(s, _addr(out)), "hmi_get_mixture")


def hmi_export_background(s: int, S=None, Q=None, vmin=None, vmax=None, lo=None, hi=None):
    """Returns (syref, n); fills whichever arrays are given."""
    sy, n = ctypes.c_uint64(), ctypes.c_int()
    _check(load().hmi_export_background(s, _addr(S), _addr(Q), _addr(vmin), _addr(vmax), _addr(lo),
                                        _addr(hi), ctypes.byref(sy), ctypes.byref(n)),
           "hmi_export_background")
    return sy.value, n.value


def hmi_import_background(s: int, S, Q, vmin, vmax, n: int, syref: int) -> None:
    _check(load().hmi_import_background(s, _addr(S), _addr(Q), _addr(vmin), _addr(vmax), n, syref),
           "hmi_import_background")


def hmi_get_last_gain(s: int) -> int:
    g = ctypes.c_uint32()
    _check(load().hmi_get_last_gain(s, ctypes.byref(g)), "hmi_get_last_gain")
    return g.value


def hmi_stream_device_bytes(w: int, h: int, params: hmi_params | None = None) -> int:
    return load().hmi_stream_device_bytes(w, h, ctypes.byref(params) if params is not None else None)


def hmi_frame_gain_noalloc(frame, w: int, h: int, syref: int, gain_min_q16: int,
                           gain_max_q16: int, gain_out, cuda_stream: int) -> None:
    """Gain of one device frame into gain_out (device uint32) using only the
    library's built-in scratch: for callers that cannot allocate device memory."""
    _check(load().hmi_frame_gain_noalloc(_addr(frame), w, h, syref, gain_min_q16, gain_max_q16,
                                         _addr(gain_out), cuda_stream), "hmi_frame_gain_noalloc")


def hmi_server_create(device_budget_bytes: int, max_queue: int = 8) -> int:
    v = load().hmi_server_create(device_budget_bytes, max_queue)
    if not v:
        raise HmiError(load().hmi_last_error(), "hmi_server_create")
    return v


def hmi_server_destroy(v: int) -> None:
    load().hmi_server_destroy(v)


def hmi_server_admit(v: int, w: int, h: int, params: hmi_params | None, learn_frames, n: int) -> int:
    """Returns the stream id; raises HmiError(HMI_ERR_NO_MEMORY) when refused.
    learn_frames None: the stream's first n submitted frames are its learning
    frames (their results carry status HMI_LEARNING)."""
    sid = ctypes.c_int()
    _check(load().hmi_server_admit(v, w, h, ctypes.byref(params) if params is not None else None,
                                   _addr(learn_frames), n, ctypes.byref(sid)), "hmi_server_admit")
    return sid.value


def hmi_server_release(v: int, stream_id: int) -> None:
    _check(load().hmi_server_release(v, stream_id), "hmi_server_release")


def hmi_server_submit(v: int, stream_id: int, frame, tag: int) -> int:
    """Returns the status (HMI_ERR_NO_MEMORY when the stream's queue is full)."""
    return load().hmi_server_submit(v, stream_id, _addr(frame), tag)


def hmi_server_submit_ref(v: int, stream_id: int, frame, tag: int) -> int:
    """By reference: `frame` must stay valid until its result is polled."""
    return load().hmi_server_submit_ref(v, stream_id, _addr(frame), tag)


def hmi_server_poll(v: int, buf: "ctypes.Array", wait_us: int) -> int:
    n = load().hmi_server_poll(v, buf, len(buf), wait_us)
    if n < 0:
        raise HmiError(n, "hmi_server_poll")
    return n


def hmi_server_stats(v: int) -> tuple[int, int, int]:
    b, t, f = ctypes.c_size_t(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().hmi_server_stats(v, ctypes.byref(b), ctypes.byref(t), ctypes.byref(f)), "hmi_server_stats")
    return b.value, t.value, f.value


def hmi_server_now_ns() -> int:
    return load().hmi_server_now_ns()


def hmi_server_rounds(v: int, max_rounds: int = 16384) -> np.ndarray:
    """The dispatcher's most recent rounds (oldest first) as a structured array."""
    buf = (hmi_server_round * max_rounds)()
    n = load().hmi_server_rounds(v, buf, max_rounds)
    if n < 0:
        raise HmiError(n, "hmi_server_rounds")
    dt = np.dtype([(k, np.dtype(t._type_)) for k, t in hmi_server_round._fields_])
    return np.frombuffer(bytes(buf)[: n * ctypes.sizeof(hmi_server_round)], dtype=dt).copy()


def hmi_last_error() -> int:
    return load().hmi_last_error()


def hmi_status_string(status: int) -> str:
    return load().hmi_status_string(status).decode()


# --------------------------------------------------------------------------- #
# Convenience object over the same calls                                      #
# --------------------------------------------------------------------------- #
class Stream:
    """One camera stream: ``learn(frames)`` once, then ``process(frame)``."""

    def __init__(self, w: int, h: int, **params):
        self.w, self.h = int(w), int(h)
        self.params = hmi_default_params(**params)
        self.handle = hmi_create_stream(self.w, self.h, self.params)

    def close(self) -> None:
        if self.handle:
            hmi_destroy_stream(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def learn(self, frames) -> None:
        n = frames.shape[0]
        hmi_learn_background(self.handle, frames, n)

    def process(self, frame, mask: bool = True):
        """Host round trip: returns (mask uint8 (h, w) or None, pointer dict)."""
        m = np.empty((self.h, self.w), np.uint8) if mask else None
        p = hmi_pointer()
        hmi_process_frame(self.handle, frame, m, p)
        return m, p.as_dict()

    def labels(self) -> np.ndarray:
        out = np.empty((self.h, self.w), np.int32)
        hmi_get_labels(self.handle, out)
        return out

    def set_interface(self, ui: hmi_interface) -> None:
        hmi_set_interface(self.handle, ui)

    def event(self) -> dict:
        return hmi_get_event(self.handle)

    def band(self) -> tuple[np.ndarray, np.ndarray]:
        lo = np.empty((self.h, self.w, 3), np.uint8)
        hi = np.empty((self.h, self.w, 3), np.uint8)
        hmi_get_band(self.handle, lo, hi)
        return lo, hi

    def mixture(self) -> np.ndarray:
        """The Gaussian mixture (bg_model 1) as (6 mix_k, h*w) uint16 planes:
        W[k], M[k][c], V[k], C[k]."""
        k = self.params.mix_k
        out = np.empty((6 * k, self.h * self.w), np.uint16)
        hmi_get_mixture(self.handle, out)
        return out

    def stats(self):
        mean = np.empty((self.h, self.w, 3), np.float32)
        std = np.empty((self.h, self.w, 3), np.float32)
        hmi_get_background_stats(self.handle, mean, std)
        return mean, std

    def last_gain(self) -> int:
        return hmi_get_last_gain(self.handle)

    def export(self) -> dict:
        shp = (self.h, self.w, 3)
        out = dict(S=np.empty(shp, np.uint32), Q=np.empty(shp, np.uint32),
                   vmin=np.empty(shp, np.uint8), vmax=np.empty(shp, np.uint8),
                   lo=np.empty(shp, np.uint8), hi=np.empty(shp, np.uint8))
        out["syref"], out["n"] = hmi_export_background(self.handle, **out)
        return out

    def import_background(self, S, Q, vmin, vmax, n: int, syref: int) -> None:
        c = np.ascontiguousarray
        hmi_import_background(self.handle, c(S, np.uint32), c(Q, np.uint32), c(vmin, np.uint8),
                              c(vmax, np.uint8), n, syref)
