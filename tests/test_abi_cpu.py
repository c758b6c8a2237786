"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function that include/hmi.h declares, and its pure host calls behave."""
import ctypes
import os
import re

import pytest

from paper_1907_04393_gb300 import hmi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hmi.h")).read()
    return sorted(set(re.findall(r"HMI_API[^;(]*?\b(hmi_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = hmi.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in hmi.h but not exported"
    assert set(names) == set(hmi.SIGNATURES), "binding and header disagree"


def test_struct_layouts():
    assert ctypes.sizeof(hmi.hmi_params) == 40
    assert ctypes.sizeof(hmi.hmi_pointer) == 40
    assert ctypes.sizeof(hmi.hmi_server_result) == 72
    assert ctypes.sizeof(hmi.hmi_server_round) == 56
    assert ctypes.sizeof(hmi.hmi_tuning) == 36
    assert ctypes.sizeof(hmi.hmi_interface) == 4 + 16 * 20 + 6 * 4
    assert ctypes.sizeof(hmi.hmi_event) == 32


def test_defaults_and_status_strings():
    p = hmi.hmi_default_params()
    assert (p.gray_tol, p.hue_lo, p.hue_hi, p.bg_margin, p.bg_k_num, p.bg_k_den) == (15, 1472, 256, 2, 5, 2)
    assert (p.open_iters, p.close_iters, p.gain_min_q16, p.gain_max_q16) == (1, 1, 32768, 131072)
    assert (p.min_area, p.click_on_pct, p.click_off_pct, p.click_window) == (50, 80, 90, 30)
    assert (p.relearn_frames, p.relearn_min, p.relearn_period, p.track_max_dist) == (0, 0, 0, 0)
    # the oracle's defaults are the library's
    import oracle
    for k, v in oracle.DEFAULTS.items():
        assert getattr(p, k) == v, k
    assert hmi.hmi_status_string(0) == "ok"
    for st in (-1, -2, -3, -4, -5):
        assert hmi.hmi_status_string(st) not in ("ok", "unknown status")
    assert hmi.load().hmi_default_params(None) == hmi.HMI_ERR_INVALID_ARG
    assert hmi.hmi_last_error() == hmi.HMI_ERR_INVALID_ARG


def test_device_bytes_accounting():
    b320 = hmi.hmi_stream_device_bytes(320, 240)
    b640 = hmi.hmi_stream_device_bytes(640, 480)
    assert 0 < b320 < b640
    assert 3.5 < b640 / b320 < 4.5
    assert hmi.hmi_stream_device_bytes(0, 10) == 0
    assert hmi.hmi_stream_device_bytes(8193, 10) == 0
    bad = hmi.hmi_default_params(hue_lo=1536)
    assert hmi.hmi_stream_device_bytes(32, 32, bad) == 0
    bad = hmi.hmi_default_params(bg_k_den=0)
    assert hmi.hmi_stream_device_bytes(32, 32, bad) == 0
    bad = hmi.hmi_default_params(open_iters=9, close_iters=8)
    assert hmi.hmi_stream_device_bytes(32, 32, bad) == 0
    # re-learning: consistent window parameters, and its sums cost device memory
    for over in (dict(relearn_frames=5, relearn_min=0, relearn_period=10),
                 dict(relearn_frames=5, relearn_min=6, relearn_period=10),
                 dict(relearn_frames=5, relearn_min=2, relearn_period=4)):
        assert hmi.hmi_stream_device_bytes(32, 32, hmi.hmi_default_params(**over)) == 0, over
    rl = hmi.hmi_default_params(relearn_frames=5, relearn_min=3, relearn_period=10)
    assert hmi.hmi_stream_device_bytes(320, 240, rl) >= b320 + 320 * 240 * 25
    # the Gaussian mixture: valid parameters only, 12 bytes per pixel and component
    for over in (dict(bg_model=2), dict(bg_model=1, mix_k=0), dict(bg_model=1, mix_k=5),
                 dict(bg_model=1, mix_bg_pct=0), dict(bg_model=1, mix_bg_pct=101),
                 dict(bg_model=1, mix_sigma0=0), dict(bg_model=1, mix_sigma0=64),
                 dict(bg_model=1, mix_sigma_min=0), dict(bg_model=1, mix_sigma_min=16),
                 dict(bg_model=1, mix_rate_n=0), dict(bg_model=1, bg_k_num=0),
                 dict(bg_model=1, relearn_frames=5, relearn_min=3, relearn_period=10),
                 dict(mix_pad=1)):
        assert hmi.hmi_stream_device_bytes(32, 32, hmi.hmi_default_params(**over)) == 0, over
    for k in (1, 2, 3, 4):
        mx = hmi.hmi_default_params(bg_model=1, mix_k=k)
        assert hmi.hmi_stream_device_bytes(320, 240, mx) >= b320 + 320 * 240 * 12 * k
    assert hmi.hmi_stream_device_bytes(32, 32, hmi.hmi_default_params(bg_model=0, mix_k=0)) > 0


def test_invalid_arguments_fail_on_host():
    lib = hmi.load()
    assert lib.hmi_learn_background(None, None, 1) == hmi.HMI_ERR_INVALID_ARG
    assert lib.hmi_process_frame(None, None, None, None) == hmi.HMI_ERR_INVALID_ARG
    assert lib.hmi_process_batch(None, 0, None, None, None) == hmi.HMI_ERR_INVALID_ARG
    assert lib.hmi_create_stream(0, 5, None) is None
    assert hmi.hmi_last_error() == hmi.HMI_ERR_INVALID_ARG
    assert lib.hmi_batch_create(None, 1) is None


def test_create_without_gpu_reports_an_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert hmi.load().hmi_create_stream(64, 48, None) is None
    assert hmi.hmi_last_error() in (hmi.HMI_ERR_DEVICE, hmi.HMI_ERR_NO_MEMORY)


def test_status_constants_match_header():
    import re
    text = open(os.path.join(ROOT, "include", "hmi.h")).read()
    found = dict((k, int(v)) for k, v in re.findall(r"#define (HMI_[A-Z_]+) \(?(-?\d+)\)?", text))
    names = [k for k in dir(hmi) if re.fullmatch(r"HMI_(OK|ERR_[A-Z_]+|LEARNING|TICK_KERNELS|MAX_ZONES)", k)]
    assert found and set(found) == set(names)
    for k in names:
        assert getattr(hmi, k) == found[k], k


def test_autotune_cache_roundtrip(tmp_path, monkeypatch):
    """The cache module stores a searched launch shape under its key and applies
    it on the next call without searching (library calls faked on the CPU)."""
    from paper_1907_04393_gb300 import autotune
    calls = {"search": 0, "set": []}

    def fake_search(b, frames, ticks, pipelined):
        calls["search"] += 1
        return {"piece_chunks": 256, "luma_ctas_per_sm": 0, "skin_ctas_per_sm": 8,
                "cc_ctas_per_sm": 4, "groups": 1, "pipeline_depth": 3}, 99.5

    monkeypatch.setattr(hmi, "hmi_batch_autotune", fake_search)
    monkeypatch.setattr(hmi, "hmi_batch_set_tuning", lambda b, t: calls["set"].append(dict(t)))
    path = str(tmp_path / "cache.json")
    shapes = [(640, 480), (320, 240), (320, 240)]
    a = autotune.tune(1, shapes, None, "GB300", True, cache_path=path)
    assert not a["cached"] and calls["search"] == 1
    b = autotune.tune(1, list(reversed(shapes)), None, "GB300", True, cache_path=path)
    assert b["cached"] and calls["search"] == 1 and calls["set"][-1]["cc_ctas_per_sm"] == 4
    c = autotune.tune(1, shapes, None, "GB300", False, cache_path=path)
    assert not c["cached"] and calls["search"] == 2
    assert a["key"] != c["key"] and autotune.key("GB300", shapes, True) == a["key"]


def test_pointer_arrays_built_once_are_passed_through():
    """A batch call given the array of buffer addresses that ptr_array built
    uses it as it is; given buffers, it builds the same addresses itself."""
    import ctypes
    import numpy as np
    from paper_1907_04393_gb300 import hmi
    bufs = [np.zeros(64, np.uint8), np.zeros(32, np.uint8)]
    arr = hmi.ptr_array(bufs)
    assert isinstance(arr, ctypes.Array) and hmi._ptr_array(arr) is arr
    assert list(arr) == [b.ctypes.data for b in bufs] == list(hmi._ptr_array(bufs))
