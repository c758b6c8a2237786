"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Bar: masks, labels, blob area and box bit-exact; gain exact; background
mean/std and pointer centroid within 1e-5 relative (FP32; in practice they are
equal, each being one correctly rounded IEEE operation on exact integers).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1907_04393_gb300 import hmi, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5
SKIN = (200, 120, 90)     # hue 70 units, chroma 110: skin for the default arc
GRAY = (128, 128, 128)
RNG = np.random.default_rng(1907)


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_pointer(pg: dict, po: dict, what=""):
    for k in ("valid", "click", "area", "x0", "y0", "x1", "y1", "label"):
        assert pg[k] == po[k], f"{what} pointer.{k}: gpu {pg[k]} oracle {po[k]}"
    for k in ("x", "y"):
        assert pg[k] == pytest.approx(po[k], rel=RTOL, abs=1e-6), f"{what} pointer.{k}"


def check_frame(g: hmi.Stream, o: oracle.OracleStream, frame: np.ndarray, dev=False, what=""):
    src = _dev(frame) if dev else frame
    m_g, p_g = g.process(src)
    l_g = g.labels()
    m_o, l_o, p_o, gain_o = o.process(frame)
    assert g.last_gain() == gain_o, f"{what} gain"
    if not np.array_equal(m_g, m_o):
        bad = np.argwhere(m_g != m_o)
        raise AssertionError(f"{what} mask differs at {len(bad)} px, first {bad[:5].tolist()}")
    if not np.array_equal(l_g, l_o):
        bad = np.argwhere(l_g != l_o)
        raise AssertionError(f"{what} labels differ at {len(bad)} px, first {bad[:5].tolist()}")
    assert_pointer(p_g, p_o, what)
    return p_g


def pair(w, h, **params):
    return hmi.Stream(w, h, **params), oracle.OracleStream(w, h, **params)


def learn_both(g, o, frames, dev=False):
    g.learn(_dev(frames) if dev else frames)
    o.learn(frames)


def black_background(g, o, gain=65536):
    """Background band [0, delta]: every non-black pixel is foreground for the
    background test; gain pinned to `gain` via the clamp."""
    shp = (g.h, g.w, 3)
    z32 = np.zeros(shp, np.uint32)
    z8 = np.zeros(shp, np.uint8)
    g.import_background(z32, z32, z8, z8, 1, 0)
    o.set_background(z32, z32, z8, z8, 1, 0)


def pattern_frame(pat: np.ndarray) -> np.ndarray:
    f = np.empty(pat.shape + (3,), np.uint8)
    f[...] = GRAY
    f[pat.astype(bool)] = SKIN
    return f


# --------------------------------------------------------------------------- #
# Learning: statistics and band                                                #
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("w,h,n", [(320, 240, 30), (37, 29, 5), (1, 1, 3), (100, 3, 1), (33, 65, 17)])
def test_learned_stats_and_band(w, h, n):
    frames = RNG.integers(0, 256, size=(n, h, w, 3), dtype=np.uint8)
    if w == 320:
        frames = synth.learn_frames(1)
    g, o = pair(w, h)
    learn_both(g, o, frames)
    mean_g, std_g = g.stats()
    mean_o, std_o = o.stats()
    np.testing.assert_allclose(mean_g, mean_o, rtol=RTOL)
    np.testing.assert_allclose(std_g, std_o, rtol=RTOL, atol=1e-6)
    ex = g.export()
    assert np.array_equal(ex["S"], o.S) and np.array_equal(ex["Q"], o.Q)
    assert np.array_equal(ex["vmin"], o.vmin) and np.array_equal(ex["vmax"], o.vmax)
    assert np.array_equal(ex["lo"], o.lo) and np.array_equal(ex["hi"], o.hi)
    assert ex["syref"] == o.syref and ex["n"] == n
    g.close()


@pytest.mark.parametrize("kn,kd,delta", [(0, 1, 0), (5, 2, 2), (15, 1, 0), (1, 15, 7), (3, 1, 255)])
def test_band_parameters(kn, kd, delta):
    frames = RNG.integers(0, 256, size=(9, 40, 48, 3), dtype=np.uint8)
    frames[:, :20] = RNG.integers(100, 110, size=(9, 20, 48, 3), dtype=np.uint8)
    g, o = pair(48, 40, bg_k_num=kn, bg_k_den=kd, bg_margin=delta)
    learn_both(g, o, frames, dev=True)
    ex = g.export()
    assert np.array_equal(ex["lo"], o.lo) and np.array_equal(ex["hi"], o.hi)
    g.close()


# --------------------------------------------------------------------------- #
# Per-pixel stages on the whole colour cube                                    #
# --------------------------------------------------------------------------- #
def _cube():
    v = np.arange(256, dtype=np.uint8)
    r, gg, b = np.meshgrid(v, v, v, indexing="ij")
    return np.stack([r, gg, b], -1).reshape(4096, 4096, 3)


@pytest.mark.parametrize("gain,tol,hue_lo,hue_hi", [(65536, 15, 1472, 256), (65536, 0, 100, 900),
                                                    (50000, 40, 1500, 20), (90000, 1, 0, 1535),
                                                    (131072, 9, 700, 700)])
def test_exhaustive_colour_cube(gain, tol, hue_lo, hue_hi):
    cube = _cube()
    kw = dict(gain_min_q16=gain, gain_max_q16=gain, gray_tol=tol, hue_lo=hue_lo, hue_hi=hue_hi,
              open_iters=0, close_iters=0, bg_margin=0)
    g, o = pair(4096, 4096, **kw)
    black_background(g, o)
    m_g, _ = g.process(_dev(cube))
    assert g.last_gain() == gain
    corr = oracle.apply_gain(cube, gain)
    z = np.zeros_like(cube)
    _, _, _, raw = oracle.fg(corr, z, z, tol, hue_lo, hue_hi)
    assert np.array_equal(m_g, raw)
    g.close()


# --------------------------------------------------------------------------- #
# Morphology and components on designed masks                                  #
# --------------------------------------------------------------------------- #
SIZES = [(1, 1), (40, 1), (1, 40), (31, 33), (32, 32), (33, 31), (64, 64), (97, 65), (257, 129),
         (300, 200), (1000, 37), (37, 1000)]


@pytest.mark.parametrize("w,h", SIZES)
@pytest.mark.parametrize("oi,ci", [(0, 0), (1, 1), (2, 0), (0, 3)])
def test_random_masks(w, h, oi, ci):
    g, o = pair(w, h, open_iters=oi, close_iters=ci, gain_min_q16=65536, gain_max_q16=65536,
                min_area=1)
    black_background(g, o)
    for p in (0.1, 0.45, 0.6, 0.9):
        pat = (RNG.random((h, w)) < p).astype(np.uint8)
        check_frame(g, o, pattern_frame(pat), dev=(w % 16 == 0), what=f"{w}x{h} p={p}")
    g.close()


def _spiral(n):
    sp = np.zeros((n, n), np.uint8)
    y, x, dy, dx, L = n // 2, n // 2, 0, 1, 1
    sp[y, x] = 1
    while L <= n:
        for _ in range(2):
            for _ in range(L):
                y, x = y + dy, x + dx
                if 0 <= y < n and 0 <= x < n:
                    sp[y, x] = 1
            dy, dx = dx, -dy
        L += 2
    return sp


def _structured(h, w):
    yy, xx = np.mgrid[0:h, 0:w]
    pats = {
        "empty": np.zeros((h, w), np.uint8),
        "full": np.ones((h, w), np.uint8),
        "checker": ((yy + xx) % 2).astype(np.uint8),
        "grid2": ((yy % 2 == 0) & (xx % 2 == 0)).astype(np.uint8),
        "diag": ((yy - xx) % 32 == 0).astype(np.uint8),
        "antidiag": ((yy + xx) % 31 == 0).astype(np.uint8),
        "hstripes": (yy % 3 == 0).astype(np.uint8),
        "vstripes": (xx % 5 == 1).astype(np.uint8),
        "corners": np.zeros((h, w), np.uint8),
        "blockcorner": (((yy % 32 == 31) & (xx % 32 == 31)) | ((yy % 32 == 0) & (xx % 32 == 0))).astype(np.uint8),
        "blockcorner2": (((yy % 32 == 31) & (xx % 32 == 0)) | ((yy % 32 == 0) & (xx % 32 == 31))).astype(np.uint8),
    }
    c = pats["corners"]
    c[0, 0] = c[0, w - 1] = c[h - 1, 0] = c[h - 1, w - 1] = 1
    sp = _spiral(max(h, w))[:h, :w]
    pats["spiral"] = sp
    u = np.zeros((h, w), np.uint8)
    u[3:h - 3, 5] = 1
    u[3:h - 3, w - 6] = 1
    u[h - 4, 5:w - 5] = 1
    pats["ushape"] = u
    return pats


@pytest.mark.parametrize("w,h", [(96, 96), (130, 70), (64, 33)])
def test_structured_masks(w, h):
    g, o = pair(w, h, open_iters=0, close_iters=0, gain_min_q16=65536, gain_max_q16=65536,
                min_area=1)
    black_background(g, o)
    for name, pat in _structured(h, w).items():
        check_frame(g, o, pattern_frame(pat), what=f"{name} {w}x{h}")
    g.close()


def test_ellipse_pointer_exact():
    w, h = 640, 480
    g, o = pair(w, h, open_iters=1, close_iters=1, gain_min_q16=65536, gain_max_q16=65536)
    black_background(g, o)
    yy, xx = np.mgrid[0:h, 0:w]
    # away from the image border, where opening keeps the shape symmetric
    for cx, cy, a, b in [(320, 240, 50, 70), (100.5, 60.5, 20, 30), (560, 400, 39.5, 60.2)]:
        pat = ((((xx - cx) / a) ** 2 + ((yy - cy) / b) ** 2) <= 1).astype(np.uint8)
        p = check_frame(g, o, pattern_frame(pat), what="ellipse")
        assert p["x"] == cx and p["y"] == cy
    g.close()


# --------------------------------------------------------------------------- #
# The synthetic workloads                                                      #
# --------------------------------------------------------------------------- #
def test_config1_all_frames():
    g, o = pair(*synth.shape(1))
    learn_both(g, o, synth.learn_frames(1))
    for t in range(synth.RUN_FRAMES[1]):
        check_frame(g, o, synth.run_frame(1, 0, t), dev=(t % 2 == 0), what=f"cfg1 t={t}")
    g.close()


def test_config2_click_sequence():
    g, o = pair(*synth.shape(2))
    learn_both(g, o, synth.learn_frames(2), dev=True)
    clicks = []
    for t in range(0, 90):
        p = check_frame(g, o, synth.run_frame(2, 0, t), dev=True, what=f"cfg2 t={t}")
        clicks.append(p["click"])
    assert 0 < sum(clicks) < len(clicks)
    g.close()


def test_config3_full_hd_contiguous():
    """The 1920x1080 stream over 120 contiguous frames (so that the click
    state and its reference-area history of a long full-HD sequence are
    compared frame by frame), then two late frames of the 600."""
    g, o = pair(*synth.shape(3))
    learn_both(g, o, synth.learn_frames(3), dev=True)
    valid = 0
    for t in list(range(120)) + [333, 599]:
        p = check_frame(g, o, synth.run_frame(3, 0, t), dev=True, what=f"cfg3 t={t}")
        valid += p["valid"]
    assert valid > 100
    g.close()


def _batch_streams(cfg, idx):
    gs, os_ = [], []
    for i in idx:
        w, h = synth.shape(cfg, i)
        g, o = pair(w, h)
        lf = synth.learn_frames(cfg, i)
        learn_both(g, o, lf, dev=True)
        gs.append(g)
        os_.append(o)
    return gs, os_


def _compare_batch(gs, os_, frames, masks_g, ptrs_g, what):
    for i, (g, o) in enumerate(zip(gs, os_)):
        m_o, l_o, p_o, _ = o.process(frames[i])
        m_g = masks_g[i].cpu().numpy() if hasattr(masks_g[i], "cpu") else masks_g[i]
        assert np.array_equal(m_g, m_o), f"{what} stream {i} mask"
        assert np.array_equal(g.labels(), l_o), f"{what} stream {i} labels"
        assert_pointer(ptrs_g[i], p_o, f"{what} stream {i}")


@pytest.mark.parametrize("fused", [1, 0, 2])
def test_batch_config4_sync_async_graph(fused):
    """64 mixed-resolution streams in one launch per tick (the persistent tick)
    or one launch per stage (the chain of kernels); each stream's result
    equals its result alone (the oracle processes every stream alone)."""
    n = synth.num_streams(4)
    gs, os_ = _batch_streams(4, range(n))
    handles = [g.handle for g in gs]
    b = hmi.hmi_batch_create(handles)
    try:
        hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), fused=fused, groups=0))
        assert hmi.hmi_batch_get_groups(b) == (1 if fused else 2)
        for t in range(4):
            frames = [synth.run_frame(4, i, t) for i in range(n)]
            mode = ("sync", "async", "graph", "graph")[t]
            if mode == "sync":
                masks = [np.empty((g.h, g.w), np.uint8) for g in gs]
                ptrs = np.zeros(n, hmi.POINTER_DTYPE)
                hmi.hmi_batch_process(b, frames, masks, ptrs)
                plist = [dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[i]])) for i in range(n)]
            else:
                dframes = [_dev(f) for f in frames]
                dmasks = [torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in gs]
                dptrs = torch.zeros(n * 40, dtype=torch.uint8, device="cuda")
                s = torch.cuda.current_stream()
                hmi.hmi_batch_process_async(b, dframes, dmasks, dptrs.data_ptr(), s.cuda_stream,
                                            mode == "graph")
                torch.cuda.synchronize()
                masks = dmasks
                arr = dptrs.cpu().numpy().view(hmi.POINTER_DTYPE)
                plist = [dict(zip(arr.dtype.names, [x.item() for x in arr[i]])) for i in range(n)]
            _compare_batch(gs, os_, frames, masks, plist, f"cfg4 t={t} {mode}")
    finally:
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()


def _pinned(a: np.ndarray, offset: int = 0):
    """A page-locked host copy of `a`, starting `offset` bytes into its buffer."""
    buf = torch.empty(a.nbytes + 64, dtype=torch.uint8).pin_memory()
    base = (-buf.data_ptr()) % 16 + offset
    view = buf[base:base + a.nbytes]
    view.numpy()[:] = a.reshape(-1)
    return view


def test_batch_pinned_host_frames():
    """Frames in page-locked host memory, aligned and misaligned, through the
    synchronous batch form; an asynchronous call with a misaligned host frame
    is refused; every result equals the oracle's."""
    idx = [0, 20, 33, 50, 61, 63]
    gs, os_ = _batch_streams(4, idx)
    b = hmi.hmi_batch_create([g.handle for g in gs])
    try:
        for t in range(2):
            frames = [synth.run_frame(4, i, t) for i in idx]
            pins = [_pinned(f, offset=(1 if (k == 2 and t == 1) else 0)) for k, f in enumerate(frames)]
            masks = [np.empty((g.h, g.w), np.uint8) for g in gs]
            ptrs = np.zeros(len(idx), hmi.POINTER_DTYPE)
            hmi.hmi_batch_process(b, pins, masks, ptrs)
            plist = [dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[i]])) for i in range(len(idx))]
            _compare_batch(gs, os_, frames, masks, plist, f"pinned t={t}")
        dmasks = [torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in gs]
        with pytest.raises(hmi.HmiError) as e:
            hmi.hmi_batch_process_async(b, pins, dmasks, None, torch.cuda.current_stream().cuda_stream, False)
        assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    finally:
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()


@pytest.mark.parametrize("mode", ["async", 2, 3])
def test_pinned_host_frames_in_stream_ordered_ticks(mode):
    """Pinned host frames given to the asynchronous and pipelined forms are read
    by the luma pass over the host link into per-phase staging frames; masks
    and pointers equal those of a twin batch given the same frames in device
    memory, tick by tick (consecutive ticks in flight use distinct staging)."""
    idx = [0, 20, 33, 50, 61]
    T = 7
    frames = [[synth.run_frame(4, i, t) for i in idx] for t in range(T)]
    pins = [[_pinned(f) for f in fr] for fr in frames]
    devs = [[_dev(f) for f in fr] for fr in frames]
    s = torch.cuda.current_stream().cuda_stream
    out = {}
    for name, src in (("pinned", pins), ("device", devs)):
        gs, _ = _batch_streams(4, idx)
        b = hmi.hmi_batch_create([g.handle for g in gs])
        hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), groups=1,
                                         pipeline_depth=mode if mode != "async" else 2))
        res = []
        for t in range(T):
            m = [torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in gs]
            p = torch.zeros(len(idx) * 40, dtype=torch.uint8, device="cuda")
            if mode == "async":
                hmi.hmi_batch_process_async(b, src[t], m, p.data_ptr(), s, t % 2 == 0)
            else:
                hmi.hmi_batch_process_pipelined(b, src[t], m, p.data_ptr(), s, t % 2 == 0)
            res.append((m, p))
        hmi.hmi_batch_flush(b, s)
        torch.cuda.synchronize()
        out[name] = [([x.cpu().numpy() for x in m], p.cpu().numpy()) for m, p in res]
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()
    for t in range(T):
        assert np.array_equal(out["pinned"][t][1], out["device"][t][1]), (mode, t)
        for k in range(len(idx)):
            assert np.array_equal(out["pinned"][t][0][k], out["device"][t][0][k]), (mode, t, k)


def test_pinned_host_frames_rows_not_multiple_of_16():
    """A pinned host frame of a stream whose width is not a multiple of 16 is
    copied first in the synchronous form (results equal the oracle's) and
    refused by the asynchronous form."""
    g, o = pair(312, 40)
    lf = np.ascontiguousarray(synth.learn_frames(1, 0, 6)[:, :40, :312])
    learn_both(g, o, lf)
    b = hmi.hmi_batch_create([g.handle])
    try:
        f = np.ascontiguousarray(synth.run_frame(1, 0, 3)[:40, :312])
        pin = _pinned(f)
        masks = [np.empty((40, 312), np.uint8)]
        ptrs = np.zeros(1, hmi.POINTER_DTYPE)
        hmi.hmi_batch_process(b, [pin], masks, ptrs)
        m_o, _, p_o, _ = o.process(f)
        assert np.array_equal(masks[0], m_o)
        assert_pointer(dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[0]])), p_o, "312 wide")
        with pytest.raises(hmi.HmiError) as e:
            hmi.hmi_batch_process_async(b, [pin], None, None, torch.cuda.current_stream().cuda_stream, False)
        assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    finally:
        hmi.hmi_batch_destroy(b)
        g.close()


def test_batch_group_count_does_not_change_results():
    """The same streams processed with 1, 3 and 5 concurrent groups per tick
    give identical masks, labels and pointers (and match the oracle)."""
    idx = [0, 5, 17, 33, 40, 47, 50, 58, 61, 63, 2, 36]
    frames = {t: [synth.run_frame(4, i, t) for i in idx] for t in range(3)}
    results = {}
    for groups in (1, 3, 5):
        gs, os_ = _batch_streams(4, idx)
        b = hmi.hmi_batch_create([g.handle for g in gs])
        hmi.hmi_batch_set_groups(b, groups)
        assert hmi.hmi_batch_get_groups(b) == groups
        out = []
        for t in range(3):
            dframes = [_dev(f) for f in frames[t]]
            dmasks = [torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in gs]
            dptrs = torch.zeros(len(idx) * 40, dtype=torch.uint8, device="cuda")
            hmi.hmi_batch_process_async(b, dframes, dmasks, dptrs.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream, t % 2 == 0)
            torch.cuda.synchronize()
            arr = dptrs.cpu().numpy().view(hmi.POINTER_DTYPE)
            plist = [dict(zip(arr.dtype.names, [x.item() for x in arr[i]])) for i in range(len(idx))]
            if groups == 3:
                _compare_batch(gs, os_, frames[t], dmasks, plist, f"groups=3 t={t}")
            out.append(([m.cpu().numpy() for m in dmasks], [g.labels() for g in gs], plist))
        results[groups] = out
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()
    for groups in (3, 5):
        for t in range(3):
            for a, c in zip(results[1][t][0], results[groups][t][0]):
                assert np.array_equal(a, c)
            for a, c in zip(results[1][t][1], results[groups][t][1]):
                assert np.array_equal(a, c)
            assert results[1][t][2] == results[groups][t][2]


def test_process_batch_cached_plan():
    idx = [0, 1, 40, 50, 60]
    gs, os_ = _batch_streams(4, idx)
    handles = [g.handle for g in gs]
    for t in range(3):
        frames = [synth.run_frame(4, i, t) for i in idx]
        ptrs = np.zeros(len(idx), hmi.POINTER_DTYPE)
        masks = [np.empty((g.h, g.w), np.uint8) for g in gs]
        hmi.hmi_process_batch(handles, frames, masks, ptrs)
        plist = [dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[i]])) for i in range(len(idx))]
        _compare_batch(gs, os_, frames, masks, plist, f"process_batch t={t}")
    for g in gs:
        g.close()


# --------------------------------------------------------------------------- #
# Sizes, placements and error paths                                            #
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("w,h", [(1, 1), (1, 50), (50, 1), (17, 5), (33, 33), (100, 75), (321, 241)])
def test_ragged_sizes_full_path(w, h):
    g, o = pair(w, h, min_area=1)
    bg = RNG.integers(0, 256, size=(h, w, 3), dtype=np.uint8)
    lf = np.clip(bg[None].astype(int) + RNG.integers(-3, 4, size=(6, h, w, 3)), 0, 255).astype(np.uint8)
    learn_both(g, o, lf, dev=True)
    for t in range(4):
        f = bg.copy()
        m = RNG.random((h, w)) < 0.3
        f[m] = SKIN
        check_frame(g, o, f, dev=(t % 2 == 1), what=f"{w}x{h} t={t}")
    g.close()


def test_maximum_dimensions_properties():
    for w, h in [(8192, 40), (40, 8192), (8192, 8192)]:
        g = hmi.Stream(w, h, gain_min_q16=65536, gain_max_q16=65536, open_iters=0, close_iters=0)
        z32 = np.zeros((h, w, 3), np.uint32)
        z8 = np.zeros((h, w, 3), np.uint8)
        g.import_background(z32, z32, z8, z8, 1, 0)
        frame = np.empty((h, w, 3), np.uint8)
        frame[...] = GRAY
        m, p = g.process(_dev(frame))
        assert not m.any() and p["valid"] == 0 and p["label"] == -1
        cx, cy = w // 2, h // 2
        a, b = min(w, h) // 4, min(w, h) // 5
        y0, y1, x0, x1 = cy - b - 1, cy + b + 2, cx - a - 1, cx + a + 2
        yy, xx = np.mgrid[y0:y1, x0:x1]
        ell = (((xx - cx) / a) ** 2 + ((yy - cy) / b) ** 2) <= 1
        frame[y0:y1, x0:x1][ell] = SKIN
        m, p = g.process(_dev(frame))
        assert (p["x"], p["y"], p["area"]) == (cx, cy, int(ell.sum()))
        assert (p["x0"], p["x1"], p["y0"], p["y1"]) == (cx - a, cx + a, cy - b, cy + b)
        assert int(m.sum()) == int(ell.sum())
        g.close()


def test_errors_and_optional_outputs():
    g = hmi.Stream(64, 48)
    frame = np.zeros((48, 64, 3), np.uint8)
    with pytest.raises(hmi.HmiError) as e:
        g.process(frame)
    assert e.value.status == hmi.HMI_ERR_NOT_LEARNED
    with pytest.raises(hmi.HmiError) as e:
        hmi.hmi_create_stream(64, 48, hmi.hmi_default_params(bg_k_den=0))
    assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    with pytest.raises(hmi.HmiError):
        hmi.hmi_learn_background(g.handle, frame, 0)
    g.learn(np.stack([frame] * 2))
    hmi.hmi_process_frame(g.handle, frame, None, None)       # outputs optional
    m, p = g.process(frame)
    assert not m.any() and p["valid"] == 0
    # the same stream cannot appear twice in a batch
    with pytest.raises(hmi.HmiError):
        hmi.hmi_batch_create([g.handle, g.handle])
    g.close()


def test_checkpoint_roundtrip():
    w, h = synth.shape(1)
    a = hmi.Stream(w, h)
    a.learn(synth.learn_frames(1))
    ex = a.export()
    b = hmi.Stream(w, h)
    b.import_background(ex["S"], ex["Q"], ex["vmin"], ex["vmax"], ex["n"], ex["syref"])
    assert np.array_equal(b.export()["lo"], ex["lo"])
    for t in range(0, 20, 4):
        f = synth.run_frame(1, 0, t)
        ma, pa = a.process(f)
        mb, pb = b.process(f)
        assert np.array_equal(ma, mb) and pa == pb
    a.close()
    b.close()


@pytest.mark.parametrize("fused", [0, 1, 2])
def test_profile_counts_classification_kernel(fused):
    w, h = synth.shape(3)
    g = hmi.Stream(w, h)
    g.learn(_dev(synth.learn_frames(3, 0, 4)))
    b = hmi.hmi_batch_create([g.handle])
    hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), fused=fused))
    f = _dev(synth.run_frame(3, 0, 0))
    m = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    hmi.hmi_batch_profile(b, 5)
    s = torch.cuda.current_stream().cuda_stream
    for i in range(7):
        hmi.hmi_batch_process_async(b, [f], [m], None, s, i % 2 == 0)
    ticks, ms = hmi.hmi_batch_profile_read(b)
    assert ticks == 5 and 0 < ms / ticks < 5.0
    t2, per = hmi.hmi_batch_profile_kernels(b)
    if fused:   # one launch for the per-pixel stage: the first kernel is all of it
        assert t2 == 5 and per["luma"] == pytest.approx(ms)
        assert all(per[k] < per["luma"] for k in ("classify", "skin", "morphology"))
    else:
        assert t2 == 5 and per["classify"] == pytest.approx(ms)
        assert all(v > 0 for k, v in per.items()
                   if k not in ("mixture", "skin", "block_components", "relearn", "relearn_band"))
    hmi.hmi_batch_destroy(b)
    g.close()


@pytest.mark.parametrize("depth", [2, 3])
def test_pipelined_ticks_equal_async_ticks(depth):
    """Two identically learned sets of streams: one processed tick by tick with
    hmi_batch_process_async, the other with pipelined calls (depth stages of
    consecutive ticks side by side, graph and direct launches, an ordinary
    call in between, a final flush).  Every tick's masks and pointers agree,
    and a multi-group plan refuses pipelining."""
    idx = [0, 7, 20, 33, 41, 50, 58, 63]
    T = 9
    frames = [[_dev(synth.run_frame(4, i, t)) for i in idx] for t in range(T)]
    ga, _ = _batch_streams(4, idx)
    gb, _ = _batch_streams(4, idx)
    ba = hmi.hmi_batch_create([g.handle for g in ga])
    bb = hmi.hmi_batch_create([g.handle for g in gb])
    hmi.hmi_batch_set_groups(ba, 1)
    hmi.hmi_batch_set_tuning(bb, dict(hmi.hmi_batch_get_tuning(bb), groups=1, pipeline_depth=depth))
    s = torch.cuda.current_stream().cuda_stream

    def outs(gs):
        return ([torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in gs],
                torch.zeros(len(gs) * 40, dtype=torch.uint8, device="cuda"))

    ref, got = [], []
    for t in range(T):
        m, p = outs(ga)
        hmi.hmi_batch_process_async(ba, frames[t], m, p.data_ptr(), s, True)
        ref.append((m, p))
        m, p = outs(gb)
        if t == 5:   # an ordinary call flushes the ticks in flight first
            hmi.hmi_batch_process_async(bb, frames[t], m, p.data_ptr(), s, False)
        else:
            hmi.hmi_batch_process_pipelined(bb, frames[t], m, p.data_ptr(), s, t % 3 != 0)
        got.append((m, p))
    hmi.hmi_batch_flush(bb, s)
    torch.cuda.synchronize()
    for t in range(T):
        for k in range(len(idx)):
            assert torch.equal(ref[t][0][k], got[t][0][k]), (t, k)
        assert torch.equal(ref[t][1], got[t][1]), t
    hmi.hmi_batch_set_groups(bb, 2)
    with pytest.raises(hmi.HmiError) as e:
        hmi.hmi_batch_process_pipelined(bb, frames[0], None, None, s, False)
    assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    for b in (ba, bb):
        hmi.hmi_batch_destroy(b)
    for g in ga + gb:
        g.close()


def test_tuning_does_not_change_results():
    """A batch under an unusual launch shape (small pieces, two luma CTAs per
    SM, small skin grid, large block-component grid, three groups) matches
    the oracle; out-of-range shapes are refused."""
    idx = [1, 9, 18, 30, 39, 47, 55, 62]
    gs, os_ = _batch_streams(4, idx)
    b = hmi.hmi_batch_create([g.handle for g in gs])
    try:
        hmi.hmi_batch_set_tuning(b, {"piece_chunks": 128, "luma_ctas_per_sm": 2, "skin_ctas_per_sm": 4,
                                     "cc_ctas_per_sm": 16, "groups": 3, "pipeline_depth": 3})
        assert hmi.hmi_batch_get_tuning(b)["piece_chunks"] == 128
        assert hmi.hmi_batch_get_groups(b) == 3
        for t in range(2):
            frames = [synth.run_frame(4, i, t) for i in idx]
            masks = [np.empty((g.h, g.w), np.uint8) for g in gs]
            ptrs = np.zeros(len(idx), hmi.POINTER_DTYPE)
            hmi.hmi_batch_process(b, frames, masks, ptrs)
            plist = [dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[i]])) for i in range(len(idx))]
            _compare_batch(gs, os_, frames, masks, plist, f"tuned t={t}")
        # the persistent tick with a small grid, small pieces, a short queue
        # lag (classify items wait for the gain) and small merge CTAs; then
        # large pieces, no lag before the tail, large merge CTAs, two groups
        for shape in ({"piece_chunks": 64, "luma_ctas_per_sm": 1, "fused": 1, "queue_lag": 3,
                       "merge_threads": 256, "groups": 1},
                      {"piece_chunks": 2048, "fused": 1, "queue_lag": 1 << 20, "merge_threads": 1024,
                       "groups": 2},
                      {"piece_chunks": 96, "luma_ctas_per_sm": 1, "fused": 2, "groups": 1},
                      {"piece_chunks": 4096, "fused": 2, "groups": 2}):
            hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), **shape))
            for t in range(2, 4):
                frames = [synth.run_frame(4, i, t) for i in idx]
                masks = [np.empty((g.h, g.w), np.uint8) for g in gs]
                ptrs = np.zeros(len(idx), hmi.POINTER_DTYPE)
                hmi.hmi_batch_process(b, frames, masks, ptrs)
                plist = [dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[i]])) for i in range(len(idx))]
                _compare_batch(gs, os_, frames, masks, plist, f"persistent {shape} t={t}")
        for bad in ({"piece_chunks": 100}, {"piece_chunks": 0}, {"skin_ctas_per_sm": 0},
                    {"cc_ctas_per_sm": 33}, {"luma_ctas_per_sm": -1}, {"groups": 65},
                    {"pipeline_depth": 1}, {"pipeline_depth": 4}, {"fused": 3}, {"fused": -1},
                    {"queue_lag": -1}, {"queue_lag": (1 << 20) + 1}, {"merge_threads": 384}):
            t = dict(hmi.hmi_batch_get_tuning(b), **bad)
            with pytest.raises(hmi.HmiError) as e:
                hmi.hmi_batch_set_tuning(b, t)
            assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    finally:
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()


def test_autotune_keeps_stream_state():
    """Autotuning a batch between ticks leaves its streams' later results as
    if it had not run (click state and pointer history are restored), and
    returns a valid launch shape that is then in force."""
    idx = [2, 17, 35, 52, 60]
    T = 6
    frames = [[_dev(synth.run_frame(4, i, t)) for i in idx] for t in range(T + 1)]
    ga, _ = _batch_streams(4, idx)
    gb, _ = _batch_streams(4, idx)
    ba = hmi.hmi_batch_create([g.handle for g in ga])
    bb = hmi.hmi_batch_create([g.handle for g in gb])
    s = torch.cuda.current_stream().cuda_stream
    out = {}
    for name, b in (("a", ba), ("b", bb)):
        res = []
        for t in range(T):
            if name == "b" and t == 3:
                tuning, us = hmi.hmi_batch_autotune(b, frames[T], 4, t % 2 == 0)
                assert us > 0 and hmi.hmi_batch_get_tuning(b)["piece_chunks"] == tuning["piece_chunks"]
            p = torch.zeros(len(idx) * 40, dtype=torch.uint8, device="cuda")
            hmi.hmi_batch_process_async(b, frames[t], None, p.data_ptr(), s, False)
            res.append(p)
        torch.cuda.synchronize()
        out[name] = [r.cpu().numpy().view(hmi.POINTER_DTYPE) for r in res]
    for t in range(T):
        assert np.array_equal(out["a"][t], out["b"][t]), t
    for b in (ba, bb):
        hmi.hmi_batch_destroy(b)
    for g in ga + gb:
        g.close()


RELEARN = dict(relearn_frames=3, relearn_min=2, relearn_period=5)


def _check_band(g, o, what):
    lo, hi = g.band()
    for name, a, b in (("lo", lo, o.lo), ("hi", hi, o.hi)):
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{what} band {name} differs at {len(bad)} values, first {bad[:4].tolist()}")


@pytest.mark.parametrize("cfg,w_over", [(1, None), (2, None), (1, 312)])
def test_relearning_matches_oracle(cfg, w_over):
    """Re-learning (window of 3 frames every 5, 2 background frames needed):
    every frame's mask, labels and pointer, and the band after every frame,
    equal the oracle's (config 1 and 2 frames; a width that is not a multiple
    of 16 exercises the padded sums)."""
    w, h = synth.shape(cfg)
    if w_over:
        w = w_over
    g, o = pair(w, h, **RELEARN)
    lf = synth.learn_frames(cfg, 0, 10)[:, :, :w]
    learn_both(g, o, np.ascontiguousarray(lf))
    for t in range(16):
        f = np.ascontiguousarray(synth.run_frame(cfg, 0, t)[:, :w])
        check_frame(g, o, f, dev=t % 2 == 1, what=f"cfg{cfg} w{w} t={t}")
        _check_band(g, o, f"cfg{cfg} w{w} t={t}")
    g.close()


def test_relearning_in_batches_and_pipelines():
    """Four streams (two re-learning, two not) in one batch: plain graph ticks
    and pipelined ticks at depths 2 and 3 all match the oracle frame by frame,
    bands included."""
    idx = [0, 20, 33, 50]
    for mode in ("plain", 2, 3):
        gs, os_ = [], []
        for k, i in enumerate(idx):
            w, h = synth.shape(4, i)
            over = RELEARN if k % 2 == 0 else {}
            g, o = pair(w, h, **over)
            learn_both(g, o, synth.learn_frames(4, i, 8), dev=True)
            gs.append(g)
            os_.append(o)
        b = hmi.hmi_batch_create([g.handle for g in gs])
        hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), groups=1,
                                         pipeline_depth=mode if mode != "plain" else 2))
        s = torch.cuda.current_stream().cuda_stream
        T = 12
        frames = [[synth.run_frame(4, i, t) for i in idx] for t in range(T)]
        dframes = [[_dev(f) for f in fr] for fr in frames]
        outs = []
        for t in range(T):
            m = [torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in gs]
            p = torch.zeros(len(idx) * 40, dtype=torch.uint8, device="cuda")
            if mode == "plain":
                hmi.hmi_batch_process_async(b, dframes[t], m, p.data_ptr(), s, True)
            else:
                hmi.hmi_batch_process_pipelined(b, dframes[t], m, p.data_ptr(), s, t % 2 == 0)
            outs.append((m, p))
        hmi.hmi_batch_flush(b, s)
        torch.cuda.synchronize()
        for t in range(T):
            arr = outs[t][1].cpu().numpy().view(hmi.POINTER_DTYPE)
            for k in range(len(idx)):
                m_o, _, p_o, _ = os_[k].process(frames[t][k], want_labels=False)
                assert np.array_equal(outs[t][0][k].cpu().numpy(), m_o), (mode, t, k)
                assert_pointer(dict(zip(arr.dtype.names, [x.item() for x in arr[k]])), p_o, f"{mode} t={t} s={k}")
        for k in range(len(idx)):
            _check_band(gs[k], os_[k], f"{mode} s={k}")
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()


# --------------------------------------------------------------------------- #
# Tracking (Sec. 2: the Mouse module tracks the hand zone)                     #
# --------------------------------------------------------------------------- #
def _track_scene(t, w=96, h=48):
    f = np.zeros((h, w, 3), np.uint8)
    f[...] = GRAY
    f[10:22, 4 + 2 * t:16 + 2 * t] = SKIN          # the hand, moving right
    s = 6 + 2 * t
    f[30:30 + s // 2 + 4, 60:60 + s] = SKIN        # a distractor, growing past it
    return f


def test_tracking_matches_oracle():
    """A moving hand and a growing distractor: with tracking the pointer stays
    on the hand, frame by frame equal to the oracle; without it, the largest
    blob wins (also equal to the oracle)."""
    for dist in (30, 0):
        g, o = pair(96, 48, track_max_dist=dist, open_iters=0, close_iters=0, min_area=20,
                    gain_min_q16=65536, gain_max_q16=65536)
        black_background(g, o)
        xs = []
        for t in range(14):
            xs.append(check_frame(g, o, _track_scene(t), dev=t % 2 == 0, what=f"track{dist} t={t}")["x"])
        assert (xs[-1] < 45) == (dist > 0), xs
        g.close()


def test_tracking_with_many_components_matches_oracle():
    """Thousands of components (the general merge path, not the shared-memory
    one) with tracking on: the chosen blob equals the oracle's."""
    w, h = 640, 480
    g, o = pair(w, h, track_max_dist=200, open_iters=0, close_iters=0, min_area=3,
                gain_min_q16=65536, gain_max_q16=65536)
    black_background(g, o)
    for t in range(4):
        pat = (RNG.random((h, w)) < 0.2).astype(np.uint8)
        pat[100 + 10 * t:160 + 10 * t, 200:260] = 1    # a large blob that moves
        check_frame(g, o, pattern_frame(pat), dev=True, what=f"many t={t}")
    g.close()


def test_tracking_in_pipelined_batches():
    """Tracking streams in a batch under pipelined ticks equal the oracle."""
    idx = [0, 33, 50]
    gs, os_ = [], []
    for i in idx:
        w, h = synth.shape(4, i)
        g, o = pair(w, h, track_max_dist=64)
        learn_both(g, o, synth.learn_frames(4, i, 8), dev=True)
        gs.append(g)
        os_.append(o)
    b = hmi.hmi_batch_create([g.handle for g in gs])
    hmi.hmi_batch_set_groups(b, 1)
    s = torch.cuda.current_stream().cuda_stream
    T = 8
    frames = [[synth.run_frame(4, i, t) for i in idx] for t in range(T)]
    dframes = [[_dev(f) for f in fr] for fr in frames]
    ptrs = []
    for t in range(T):
        p = torch.zeros(len(idx) * 40, dtype=torch.uint8, device="cuda")
        hmi.hmi_batch_process_pipelined(b, dframes[t], None, p.data_ptr(), s, True)
        ptrs.append(p)
    hmi.hmi_batch_flush(b, s)
    torch.cuda.synchronize()
    for t in range(T):
        arr = ptrs[t].cpu().numpy().view(hmi.POINTER_DTYPE)
        for k in range(len(idx)):
            _, _, p_o, _ = os_[k].process(frames[t][k], want_labels=False)
            assert_pointer(dict(zip(arr.dtype.names, [x.item() for x in arr[k]])), p_o, f"t={t} s={k}")
    hmi.hmi_batch_destroy(b)
    for g in gs:
        g.close()


# --------------------------------------------------------------------------- #
# Interface module and driving wheel (Sec. 2, Sec. 4)                          #
# --------------------------------------------------------------------------- #
def test_interface_events_match_oracle():
    """Config 2 (a moving hand that opens and closes): zones on the image's
    quadrants and a wheel around its centre; every frame's event equals the
    oracle's, and bad interfaces are refused."""
    w, h = synth.shape(2)
    zones = [(0, 0, w // 2 - 1, h // 2 - 1, 11), (w // 2, 0, w - 1, h // 2 - 1, 12),
             (0, h // 2, w // 2 - 1, h - 1, 13), (w // 2, h // 2, w - 1, h - 1, 14)]
    wheel = (w // 2, h // 2, 40, 260, 64)
    g, o = pair(w, h, track_max_dist=80)
    learn_both(g, o, synth.learn_frames(2, 0, 12))
    g.set_interface(hmi.make_interface(zones, wheel))
    o.set_interface(zones, (1,) + wheel)
    seen = set()
    for t in range(0, 60, 3):
        f = synth.run_frame(2, 0, t)
        check_frame(g, o, f, dev=t % 2 == 0, what=f"t={t}")
        ev = hmi.hmi_get_event(g.handle)
        frame_no = ev.pop("frame")
        assert ev == o.event, (t, ev, o.event)
        assert frame_no == o.frames
        seen.add((ev["zone"], ev["on_wheel"]))
    assert len(seen) >= 3, seen        # the hand visits several zones and the wheel
    too_many = hmi.make_interface(zones)
    too_many.nzones = hmi.HMI_MAX_ZONES + 1
    for bad in (too_many, hmi.make_interface([], (10, 10, 50, 40, 0)),
                hmi.make_interface([], (10, 10, 5, 40, 4000))):
        with pytest.raises(hmi.HmiError):
            g.set_interface(bad)
    g.close()


# --------------------------------------------------------------------------- #
# The persistent tick (hmi_tuning.fused = 1) against the oracle                #
# --------------------------------------------------------------------------- #
def _fused_batch(gs, fused=1, **over):
    b = hmi.hmi_batch_create([g.handle for g in gs])
    hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), fused=fused, groups=1, **over))
    return b


def _batch_step(b, gs, frames, host=False):
    n = len(gs)
    if host:
        masks = [np.empty((g.h, g.w), np.uint8) for g in gs]
        ptrs = np.zeros(n, hmi.POINTER_DTYPE)
        hmi.hmi_batch_process(b, frames, masks, ptrs)
        return masks, [dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[i]])) for i in range(n)]
    dframes = [_dev(f) for f in frames]
    dmasks = [torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in gs]
    dptrs = torch.zeros(n * 40, dtype=torch.uint8, device="cuda")
    hmi.hmi_batch_process_async(b, dframes, dmasks, dptrs.data_ptr(), torch.cuda.current_stream().cuda_stream, True)
    torch.cuda.synchronize()
    arr = dptrs.cpu().numpy().view(hmi.POINTER_DTYPE)
    return [m.cpu().numpy() for m in dmasks], [dict(zip(arr.dtype.names, [x.item() for x in arr[i]])) for i in range(n)]


@pytest.mark.parametrize("fused", [1, 2])
@pytest.mark.parametrize("cfg,frames,piece", [(1, range(0, 60, 3), 64), (2, range(0, 300, 15), 512),
                                              (3, range(0, 600, 100), 1024)])
def test_persistent_tick_single_stream_configs(cfg, frames, piece, fused):
    """Single streams of the three plain configurations, one stream per
    persistent launch (every classify item waits for the stream's gain) or
    per cooperative launch (every band test waits at the grid barrier)."""
    w, h = synth.shape(cfg)
    g, o = pair(w, h)
    learn_both(g, o, synth.learn_frames(cfg), dev=True)
    b = _fused_batch([g], fused=fused, piece_chunks=piece)
    try:
        for t in frames:
            fr = synth.run_frame(cfg, 0, t)
            masks, ptrs = _batch_step(b, [g], [fr], host=(t % 2 == 1))
            m_o, l_o, p_o, gain_o = o.process(fr)
            assert g.last_gain() == gain_o, f"cfg{cfg} t={t} gain"
            assert np.array_equal(masks[0], m_o), f"cfg{cfg} t={t} mask"
            assert np.array_equal(g.labels(), l_o), f"cfg{cfg} t={t} labels"
            assert_pointer(ptrs[0], p_o, f"cfg{cfg} t={t}")
    finally:
        hmi.hmi_batch_destroy(b)
        g.close()


@pytest.mark.parametrize("fused", [1, 2])
def test_persistent_tick_ragged_sizes_pinned_and_pipelined(fused):
    """Ragged frame sizes (rows not a multiple of 16 or 32 pixels, tiny
    frames) in one persistent (or cooperative) launch, then the 16-aligned
    ones from pinned host frames (copied into staging by the luma pass) in
    pipelined calls."""
    shapes = [(1, 1), (17, 5), (33, 33), (100, 75), (321, 241), (64, 48), (320, 240), (160, 96)]
    gs, os_ = [], []
    for w, h in shapes:
        g, o = pair(w, h)
        lf = RNG.integers(0, 256, size=(3, h, w, 3), dtype=np.uint8)
        learn_both(g, o, lf, dev=True)
        gs.append(g)
        os_.append(o)
    b = _fused_batch(gs, fused=fused, piece_chunks=32, queue_lag=7)
    try:
        for t in range(3):
            frames = [RNG.integers(0, 256, size=(g.h, g.w, 3), dtype=np.uint8) for g in gs]
            masks, ptrs = _batch_step(b, gs, frames)
            for i, (g, o) in enumerate(zip(gs, os_)):
                m_o, l_o, p_o, _ = o.process(frames[i])
                assert np.array_equal(masks[i], m_o), f"{shapes[i]} t={t} mask"
                assert np.array_equal(g.labels(), l_o), f"{shapes[i]} t={t} labels"
                assert_pointer(ptrs[i], p_o, f"{shapes[i]} t={t}")
    finally:
        hmi.hmi_batch_destroy(b)
    sel = [i for i, (w, h) in enumerate(shapes) if w % 16 == 0]
    ga, oa = [gs[i] for i in sel], [os_[i] for i in sel]
    b = _fused_batch(ga, fused=fused, pipeline_depth=2)
    try:
        s = torch.cuda.current_stream().cuda_stream
        dmasks = [torch.empty((g.h, g.w), dtype=torch.uint8, device="cuda") for g in ga]
        dptrs = [torch.zeros(len(ga) * 40, dtype=torch.uint8, device="cuda") for _ in range(4)]
        pinned, expect = [], []
        for t in range(4):
            frames = [synth.run_frame(4, 3 + i, t)[:g.h, :g.w].copy() for i, g in enumerate(ga)]
            pinned.append([_pinned(f) for f in frames])
            expect.append([o.process(f) for o, f in zip(oa, frames)])
            hmi.hmi_batch_process_pipelined(b, pinned[t], dmasks if t == 3 else None, dptrs[t].data_ptr(), s, True)
        hmi.hmi_batch_flush(b, s)
        torch.cuda.synchronize()
        for t in range(4):
            arr = dptrs[t].cpu().numpy().view(hmi.POINTER_DTYPE)
            for i in range(len(ga)):
                assert_pointer(dict(zip(arr.dtype.names, [x.item() for x in arr[i]])), expect[t][i][2],
                               f"pinned pipelined t={t} stream {i}")
        for i in range(len(ga)):
            assert np.array_equal(dmasks[i].cpu().numpy(), expect[3][i][0])
            assert np.array_equal(ga[i].labels(), expect[3][i][1])
    finally:
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()
