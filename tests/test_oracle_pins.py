"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test checks one stage of the oracle against a closed form, a library
routine (colorsys, scipy.ndimage, numpy), brute force on tiny inputs, a
hand-worked fixture under tests/golden/, or the generator's ground truth, so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""
import colorsys
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from paper_1907_04393_gb300 import synth

RNG = np.random.default_rng(20190709)
EIGHT = np.ones((3, 3), bool)


# --------------------------------------------------------------------------- #
# Hue (Sec. 3.1 (iii))                                                         #
# --------------------------------------------------------------------------- #
def _golden_rows(golden_dir, name):
    rows = []
    with open(f"{golden_dir}/{name}") as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def test_hue_special_colours(golden_dir):
    for row in _golden_rows(golden_dir, "hue_special.txt"):
        r, g, b, h = map(int, row.split())
        assert oracle.hue(r, g, b) == h, (r, g, b)


def _circ_dist(a, b, period=1536.0):
    d = abs(a - b) % period
    return min(d, period - d)


def test_hue_within_half_unit_of_textbook_hsv():
    cols = RNG.integers(0, 256, size=(20000, 3))
    worst = 0.0
    for r, g, b in cols:
        h = oracle.hue(r, g, b)
        if max(r, g, b) == min(r, g, b):
            assert h == -1
            continue
        ref = colorsys.rgb_to_hsv(r / 255.0, g / 255.0, b / 255.0)[0] * 1536.0
        d = _circ_dist(h, ref)
        worst = max(worst, d)
        assert d <= 0.5 + 1e-9, (r, g, b, h, ref)
    assert worst > 0.4  # rounding is really happening (not an identity test)


def test_hue_hsl_equals_hsv():
    # HSV (Sec. 3.1 (iii) item) and HSL (its text) share the hue.
    for r, g, b in RNG.integers(0, 256, size=(2000, 3)):
        if max(r, g, b) == min(r, g, b):
            continue
        hv = colorsys.rgb_to_hsv(r / 255, g / 255, b / 255)[0]
        hl = colorsys.rgb_to_hls(r / 255, g / 255, b / 255)[0]
        assert abs(hv - hl) < 1e-12


def _cube():
    v = np.arange(256, dtype=np.uint8)
    r, g, b = np.meshgrid(v, v, v, indexing="ij")
    return np.stack([r, g, b], -1).reshape(4096, 4096, 3)


def _textbook_hue_units(c):
    """Float HSV hue * 1536 of an (..., 3) uint8 array (NaN where gray)."""
    f = c.astype(np.float64)
    r, g, b = f[..., 0], f[..., 1], f[..., 2]
    mx, mn = f.max(-1), f.min(-1)
    d = mx - mn
    with np.errstate(invalid="ignore", divide="ignore"):
        h = np.where(mx == r, (g - b) / d % 6.0,
                     np.where(mx == g, (b - r) / d + 2.0, (r - g) / d + 4.0))
    h = h * 256.0 % 1536.0
    return np.where(d == 0, np.nan, h)


def test_exhaustive_cube_integer_hue_is_rounded_textbook_hue():
    """All 2^24 colours.  256 t / d is never within 1/510 of a half-integer
    (d <= 255 cannot supply the factor 512), so rounding the float textbook
    hue gives the exact integer hue; float64 error is far below that margin."""
    c = _cube()
    h = _textbook_hue_units(c)
    defined = ~np.isnan(h)
    frac = h[defined] - np.floor(h[defined])
    assert np.abs(frac - 0.5).min() > 1.0 / 600
    expect = np.full(h.shape, -1, np.int64)
    expect[defined] = np.floor(h[defined] + 0.5).astype(np.int64) % 1536
    assert np.array_equal(oracle.hue_map(c), expect)


def _arc_table(lo, hi):
    """Members of the closed hue arc [lo, hi] modulo one turn, walked unit by unit."""
    t = np.zeros(1536, bool)
    k = lo
    while True:
        t[k] = True
        if k == hi:
            return t
        k = (k + 1) % 1536


@pytest.mark.parametrize("hue_lo,hue_hi,tol", [(1472, 256, 15), (100, 900, 0), (1500, 20, 40),
                                               (0, 1535, 1), (700, 700, 15), (0, 300, 9)])
def test_exhaustive_cube_gray_and_hue_masks(hue_lo, hue_hi, tol):
    """All 2^24 colours: fg2 against the HSV chroma (255 * S * V = max - min),
    fg3 against the rounded textbook hue looked up in the walked arc."""
    c = _cube()
    lo = np.zeros_like(c)
    hi = np.zeros_like(c)
    fg1, fg2, fg3, raw = oracle.fg(c, lo, hi, tol, hue_lo, hue_hi)
    f = c.astype(np.float64) / 255.0
    hsv_s = np.where(f.max(-1) > 0, (f.max(-1) - f.min(-1)) / np.maximum(f.max(-1), 1e-300), 0.0)
    chroma = np.rint(hsv_s * f.max(-1) * 255.0)
    assert np.array_equal(fg2, (chroma >= tol).astype(np.uint8))
    h = _textbook_hue_units(c)
    defined = ~np.isnan(h)
    hint = np.zeros(h.shape, np.int64)
    hint[defined] = np.floor(h[defined] + 0.5).astype(np.int64) % 1536
    expect = defined & _arc_table(hue_lo, hue_hi)[hint]
    assert np.array_equal(fg3, expect.astype(np.uint8))
    # fg1: a band [0, 0] keeps only pure black as background
    assert np.array_equal(fg1, (c.max(-1) > 0).astype(np.uint8))
    assert np.array_equal(raw, fg1 & fg2 & fg3)


# --------------------------------------------------------------------------- #
# Background learning (Sec. 2 FIZI init; Sec. 3.1 (i))                         #
# --------------------------------------------------------------------------- #
def test_learn_hand_worked_fixture(golden_dir):
    rows = [r.split("|") for r in _golden_rows(golden_dir, "learn_3frames.txt")]
    vals = np.array([[int(x) for x in r[0].split()] for r in rows])  # (3 ch, 3 frames)
    frames = vals.T.reshape(3, 1, 1, 3).astype(np.uint8)
    S, Q, vmin, vmax = oracle.learn_stats(frames)
    mean, std = oracle.learn_meanstd(S, Q, 3)
    lo, hi = oracle.learn_band(S, Q, vmin, vmax, 3, 5, 2, 2)
    for c, r in enumerate(rows):
        s, q, mn, mx = map(int, r[1].split())
        mu, sd = map(float, r[2].split())
        l, h = map(int, r[3].split())
        assert (S[0, 0, c], Q[0, 0, c], vmin[0, 0, c], vmax[0, 0, c]) == (s, q, mn, mx)
        assert mean[0, 0, c] == pytest.approx(mu, rel=1e-6)
        assert std[0, 0, c] == pytest.approx(sd, rel=1e-6, abs=1e-7)
        assert (lo[0, 0, c], hi[0, 0, c]) == (l, h)


def test_learn_single_frame_closed_form():
    f = RNG.integers(0, 256, size=(1, 7, 9, 3), dtype=np.uint8)
    S, Q, vmin, vmax = oracle.learn_stats(f)
    mean, std = oracle.learn_meanstd(S, Q, 1)
    assert np.array_equal(mean, f[0].astype(np.float32))
    assert not std.any()
    for delta in (0, 2, 9):
        lo, hi = oracle.learn_band(S, Q, vmin, vmax, 1, 5, 2, delta)
        v = f[0].astype(np.int32)
        assert np.array_equal(lo, np.clip(v - delta, 0, 255))
        assert np.array_equal(hi, np.clip(v + delta, 0, 255))


def test_learn_stats_against_numpy():
    f = RNG.integers(0, 256, size=(37, 5, 6, 3), dtype=np.uint8)
    S, Q, vmin, vmax = oracle.learn_stats(f)
    assert np.array_equal(S, f.astype(np.uint64).sum(0))
    assert np.array_equal(Q, (f.astype(np.uint64) ** 2).sum(0))
    assert np.array_equal(vmin, f.min(0)) and np.array_equal(vmax, f.max(0))
    mean, std = oracle.learn_meanstd(S, Q, 37)
    ff = f.astype(np.float64)
    np.testing.assert_allclose(mean, ff.mean(0), rtol=1e-6)
    np.testing.assert_allclose(std, ff.std(0), rtol=1e-5, atol=1e-5)


def test_paper_literal_band_is_min_max():
    # k = 0 and delta = 0: the band is the learned [min, max] of Sec. 3.1 (i)
    f = RNG.integers(0, 256, size=(11, 4, 5, 3), dtype=np.uint8)
    S, Q, vmin, vmax = oracle.learn_stats(f)
    lo, hi = oracle.learn_band(S, Q, vmin, vmax, 11, 0, 1, 0)
    assert np.array_equal(lo, f.min(0)) and np.array_equal(hi, f.max(0))


def test_band_edges_against_decimal_mu_minus_k_sigma():
    getcontext().prec = 60
    for _ in range(3000):
        n = int(RNG.integers(1, 200))
        spread = int(RNG.integers(0, 128))
        centre = int(RNG.integers(0, 256))
        v = np.clip(RNG.normal(centre, spread + 0.01, size=n).round(), 0, 255).astype(np.int64)
        S, Q = int(v.sum()), int((v * v).sum())
        kn, kd = int(RNG.integers(0, 16)), int(RNG.integers(1, 16))
        D = n * Q - S * S
        mu = Decimal(S) / n
        ks = Decimal(kn) / kd * Decimal(D).sqrt() / n
        lo_ref = math.floor(mu - ks)
        hi_ref = math.ceil(mu + ks)
        assert oracle.band_low(S, Q, n, kn, kd) == lo_ref, (n, S, Q, kn, kd)
        assert oracle.band_high(S, Q, n, kn, kd) == hi_ref, (n, S, Q, kn, kd)


# --------------------------------------------------------------------------- #
# Brightness (Sec. 2 brightness correction; Sec. 3.2)                          #
# --------------------------------------------------------------------------- #
def test_luma8_close_to_bt601():
    cols = RNG.integers(0, 256, size=(5000, 3)).astype(np.uint8)
    for c in cols:
        y = oracle.luma_sum(c.reshape(1, 1, 3))
        ref = 0.299 * c[0] + 0.587 * c[1] + 0.114 * c[2]
        assert abs(y - ref) <= 1.5


def test_luma8_hand_worked_fixture(golden_dir):
    """Hand-worked luma values where the rounding term of the integer luma
    decides the result, and a small frame's exact luma sum."""
    rows = [[c.strip() for c in r.split("|")] for r in _golden_rows(golden_dir, "luma_rounding.txt")]
    decided = 0
    for row in rows:
        if row[0].startswith("frame"):
            _, h, w = row[0].split()
            px = [tuple(map(int, p.split())) for line in row[1].split(";") for p in line.split(",")]
            frame = np.array(px, np.uint8).reshape(int(h), int(w), 3)
            assert oracle.luma_sum(frame) == int(row[2])
            continue
        r, g, b = map(int, row[0].split())
        assert 77 * r + 150 * g + 29 * b + 128 == int(row[1]), row   # the fixture's own arithmetic
        assert oracle.luma_sum(np.array([[[r, g, b]]], np.uint8)) == int(row[2]), row
        decided += row[3].startswith("r")
    assert decided >= 6


def test_ref_luma_is_floor_of_mean():
    f = RNG.integers(0, 256, size=(7, 9, 11, 3), dtype=np.uint8)
    sums = [oracle.luma_sum(x) for x in f]
    assert oracle.ref_luma(f) == sum(sums) // 7


def test_gain_closed_forms():
    assert oracle.gain(1000, 1000, 32768, 131072) == 65536
    assert oracle.gain(0, 5000, 32768, 131072) == 65536          # black frame
    assert oracle.gain(2000, 1000, 32768, 131072) == 32768        # exactly 0.5
    assert oracle.gain(4000, 1000, 32768, 131072) == 32768        # clamped low
    assert oracle.gain(1000, 3000, 32768, 131072) == 131072       # clamped high
    assert oracle.gain(3, 4, 0, 1 << 24) == round(4 / 3 * 65536)
    for _ in range(500):
        sy = int(RNG.integers(1 << 16, 1 << 30))
        syref = int(RNG.integers(0, 1 << 30))
        g = oracle.gain(sy, syref, 0, (1 << 32) - 1)
        assert abs(g - syref * 65536 / sy) <= 0.5 + 1e-9


def test_apply_gain_rounds_and_saturates():
    c = np.arange(256, dtype=np.uint8)
    for g in (0, 1, 32768, 65535, 65536, 65537, 98304, 131072):
        out = oracle.apply_gain(c, g).astype(np.float64)
        ref = np.minimum(255.0, c * (g / 65536.0))
        assert np.all(np.abs(out - ref) <= 0.5)
    assert np.array_equal(oracle.apply_gain(c, 65536), c)


def test_uniform_brightness_scale_is_undone():
    """All learning frames = B; run frame = round(s * B) without clipping:
    the corrected frame is within 1 of B and the whole path gives an empty mask."""
    h, w = 24, 40
    yy, xx = np.mgrid[0:h, 0:w]
    for s in (0.7, 0.85, 1.0, 1.13, 1.3):
        B = np.stack([30 + 3 * xx, 40 + 4 * yy, 150 - 2 * xx], -1).astype(np.uint8)
        B[5:12, 8:20] = (190, 140, 110)     # a skin-coloured patch in the background
        run = np.clip(np.round(B * s), 0, 255).astype(np.uint8)
        assert run.max() < 255
        o = oracle.OracleStream(w, h)
        o.learn(np.stack([B] * 4))
        mask, labels, ptr, g = o.process(run)
        corr = oracle.apply_gain(run, g).astype(int)
        assert np.abs(corr - B.astype(int)).max() <= 1, s
        assert not mask.any() and ptr["valid"] == 0 and ptr["label"] == -1


def test_frame_equal_to_learning_frame_has_no_foreground():
    f = synth.learn_frames(1, 0, 6)
    S, Q, vmin, vmax = oracle.learn_stats(f)
    lo, hi = oracle.learn_band(S, Q, vmin, vmax, 6, 5, 2, 2)
    for i in range(6):
        fg1, _, _, _ = oracle.fg(f[i], lo, hi, 15, 1472, 256)    # gain 1
        assert not fg1.any()


def test_band_edges_inclusive():
    lo = np.full((1, 4, 3), 100, np.uint8)
    hi = np.full((1, 4, 3), 120, np.uint8)
    c = np.array([[[100, 110, 120], [99, 110, 110], [110, 121, 110], [120, 120, 100]]], np.uint8)
    fg1, _, _, _ = oracle.fg(c, lo, hi, 0, 0, 1535)
    assert fg1.tolist() == [[0, 1, 1, 0]]


# --------------------------------------------------------------------------- #
# Morphology (Sec. 3.1 erosion and dilation)                                   #
# --------------------------------------------------------------------------- #
SIZES = [(1, 1), (1, 7), (6, 1), (2, 2), (5, 3), (8, 8), (13, 17), (37, 29), (33, 64)]


@pytest.mark.parametrize("h,w", SIZES)
def test_erode_dilate_against_scipy(h, w):
    for p in (0.3, 0.6, 0.9):
        m = (RNG.random((h, w)) < p).astype(np.uint8)
        e = ndi.binary_erosion(m, EIGHT, border_value=1).astype(np.uint8)
        d = ndi.binary_dilation(m, EIGHT, border_value=0).astype(np.uint8)
        assert np.array_equal(oracle.erode(m), e)
        assert np.array_equal(oracle.dilate(m), d)


@pytest.mark.parametrize("oi,ci", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 1), (1, 3)])
def test_open_close_sequence_against_scipy(oi, ci):
    m = (RNG.random((29, 41)) < 0.55).astype(np.uint8)
    ref = m.astype(bool)
    for _ in range(oi):
        ref = ndi.binary_dilation(ndi.binary_erosion(ref, EIGHT, border_value=1), EIGHT, border_value=0)
    for _ in range(ci):
        ref = ndi.binary_erosion(ndi.binary_dilation(ref, EIGHT, border_value=0), EIGHT, border_value=1)
    assert np.array_equal(oracle.morph(m, oi, ci), ref.astype(np.uint8))


def test_morphology_special_cases():
    m = np.zeros((9, 9), np.uint8)
    m[4, 4] = 1
    assert not oracle.morph(m, 1, 0).any()                      # isolated pixel opened away
    m = np.zeros((9, 12), np.uint8)
    m[2:7, 1:5] = 1
    m[2:7, 6:10] = 1                                            # 1-px gap at column 5
    assert oracle.morph(m, 0, 1)[2:7, 5].all()                  # bridged by closing
    full = np.ones((5, 6), np.uint8)
    assert oracle.erode(full).all()                             # border is neutral
    corner = np.zeros((6, 6), np.uint8)
    corner[:3, :3] = 1
    assert oracle.morph(corner, 1, 1)[:3, :3].all()             # blob on the border kept


# --------------------------------------------------------------------------- #
# Connected components (Mouse module: the hand zone)                           #
# --------------------------------------------------------------------------- #
def _check_against_scipy(m):
    lab, n = oracle.label(m)
    ref, nref = ndi.label(m, structure=EIGHT)
    assert n == nref
    assert np.array_equal(lab < 0, m == 0)
    idx = np.arange(m.size).reshape(m.shape)
    for k in range(1, nref + 1):
        sel = ref == k
        vals = np.unique(lab[sel])
        assert vals.size == 1 and vals[0] == idx[sel].min()


@pytest.mark.parametrize("h,w", SIZES + [(64, 96), (70, 33)])
def test_labels_against_scipy(h, w):
    for p in (0.2, 0.45, 0.6, 0.85):
        _check_against_scipy((RNG.random((h, w)) < p).astype(np.uint8))


def test_hand_counted_components():
    cb = (np.add.outer(np.arange(10), np.arange(12)) % 2).astype(np.uint8)
    assert oracle.label(cb)[1] == 1                                   # checkerboard
    diag = np.eye(8, dtype=np.uint8)
    assert oracle.label(diag)[1] == 1                                 # diagonal chain
    grid = np.zeros((9, 11), np.uint8)
    grid[::2, ::2] = 1
    assert oracle.label(grid)[1] == 5 * 6                             # isolated pixels
    u = np.zeros((40, 40), np.uint8)
    u[5:35, 5] = 1
    u[5:35, 34] = 1
    u[34, 5:35] = 1                                                   # U crossing 32-px tiles
    lab, n = oracle.label(u)
    assert n == 1 and lab[5, 5] == 5 * 40 + 5 and lab[5, 34] == 5 * 40 + 5
    sp = np.zeros((21, 21), np.uint8)                                 # square spiral
    y, x, dy, dx, L = 10, 10, 0, 1, 1
    sp[y, x] = 1
    while True:
        for _ in range(2):
            for _ in range(L):
                y, x = y + dy, x + dx
                if not (0 <= y < 21 and 0 <= x < 21):
                    break
                sp[y, x] = 1
            dy, dx = dx, -dy
        L += 2
        if L > 21:
            break
    assert oracle.label(sp)[1] == 1
    assert oracle.label(np.zeros((3, 3), np.uint8))[1] == 0


# --------------------------------------------------------------------------- #
# Pointer and click state (Sec. 2: pointer and its clicked state)             #
# --------------------------------------------------------------------------- #
def _ellipse(h, w, cy, cx, a, b):
    yy, xx = np.mgrid[0:h, 0:w]
    return ((((xx - cx) / a) ** 2 + ((yy - cy) / b) ** 2) <= 1.0).astype(np.uint8)


def test_ellipse_centroid_and_bbox_exact():
    for (cy, cx, a, b) in [(20, 30, 10.0, 6.0), (31.5, 40.5, 12.3, 20.1), (50, 50, 40.0, 40.0)]:
        m = _ellipse(101, 103, cy, cx, a, b)
        lab, _ = oracle.label(m)
        p = oracle.pointer_from_labels(lab, 50)
        assert p["x"] == cx and p["y"] == cy
        assert p["area"] == int(m.sum()) and p["valid"] == 1
        ys, xs = np.nonzero(m)
        assert (p["x0"], p["y0"], p["x1"], p["y1"]) == (xs.min(), ys.min(), xs.max(), ys.max())
        # closed form of the box of a pixel-centred ellipse: centre -/+ floor(semi-axis)
        if cx == int(cx) and cy == int(cy):
            assert (p["x0"], p["x1"]) == (cx - math.floor(a), cx + math.floor(a))
            assert (p["y0"], p["y1"]) == (cy - math.floor(b), cy + math.floor(b))


def test_largest_blob_and_ties():
    m = _ellipse(60, 80, 20, 20, 6, 6) | _ellipse(60, 80, 40, 60, 9, 9)
    p = oracle.pointer_from_labels(oracle.label(m)[0], 1)
    assert (p["x"], p["y"]) == (60.0, 40.0)
    m = _ellipse(60, 80, 40, 20, 7, 7) | _ellipse(60, 80, 20, 60, 7, 7)   # equal areas
    lab, _ = oracle.label(m)
    p = oracle.pointer_from_labels(lab, 1)
    assert p["label"] == min(lab[40, 20], lab[20, 60]) and (p["x"], p["y"]) == (60.0, 20.0)
    p = oracle.pointer_from_labels(oracle.label(np.zeros((4, 4), np.uint8))[0], 1)
    assert (p["valid"], p["area"], p["label"], p["x0"], p["x"]) == (0, 0, -1, -1, -1.0)
    small = np.zeros((10, 10), np.uint8)
    small[2:4, 2:4] = 1
    p = oracle.pointer_from_labels(oracle.label(small)[0], 5)
    assert p["valid"] == 0 and p["area"] == 4


def test_click_state_machine_hand_worked():
    st = oracle.ClickState(30)
    seq = [(1, 100, 0), (1, 100, 0), (1, 50, 1), (1, 60, 1), (0, 10, 1), (1, 95, 0),
           (1, 79, 1), (1, 91, 1), (1, 92, 0)]
    # hand-worked: first frame has no A_ref -> 0; 100*100 > 90*100 -> 0;
    # 5000 < 8000 -> 1; 6000 < 8000 -> 1; invalid -> unchanged; 9500 > 9000 -> 0;
    # 7900 < 8000 -> 1; 9100 > 9000 -> 0; 9200 > 9000 -> 0
    got = []
    for valid, area, _ in seq:
        p = st.update(dict(valid=valid, click=0, x=0.0, y=0.0, area=area, x0=0, y0=0, x1=0,
                           y1=0, label=0), 80, 90)
        got.append(p["click"])
    assert got == [0, 0, 1, 1, 1, 0, 1, 0, 0]
    st = oracle.ClickState(2)                              # sliding window of 2 valid frames
    out = [st.update(dict(valid=1, click=0, x=0.0, y=0.0, area=a, x0=0, y0=0, x1=0, y1=0,
                          label=0), 80, 90)["click"] for a in (100, 100, 70, 70, 70)]
    # A_ref: -,100,100,100(hist 100,70),70(hist 70,70): 7000 > 6300 -> clear
    assert out == [0, 0, 1, 1, 0]


def test_click_state_machine_strict_boundaries():
    """The click is set only when 100*area is strictly below on_pct*A_ref and
    cleared only when strictly above off_pct*A_ref: equality changes nothing."""
    def run(areas, on, off, window=30):
        st = oracle.ClickState(window)
        return [st.update(dict(valid=1, click=0, x=0.0, y=0.0, area=a, x0=0, y0=0, x1=0, y1=0,
                               label=0), on, off)["click"] for a in areas]
    # A_ref stays 100: 8000 == 80*100 keeps 0; 5000 < 8000 sets; 9000 == 90*100
    # keeps 1; 9100 > 9000 clears
    assert run([100, 80, 50, 90, 91], 80, 90) == [0, 0, 1, 1, 0]
    # one unit either side of each boundary
    assert run([100, 79], 80, 90) == [0, 1]
    assert run([100, 50, 91], 80, 90) == [0, 1, 0]
    # on and off at the same percentage: equality neither sets nor clears
    assert run([200, 150, 100, 150, 151], 75, 75) == [0, 0, 1, 1, 0]


# --------------------------------------------------------------------------- #
# Whole path against the generator's ground truth (sanity of the readings)     #
# --------------------------------------------------------------------------- #
def test_pointer_tracks_generated_hand_config1():
    o = oracle.OracleStream(*synth.shape(1))
    o.learn(synth.learn_frames(1))
    for t in range(0, 60, 7):
        _, _, p, _ = o.process(synth.run_frame(1, 0, t))
        (cx, cy, a, b), = synth.truth(1, 0, t)[0]
        assert p["valid"] == 1
        assert abs(p["x"] - cx) < 0.6 and abs(p["y"] - cy) < 0.6
        assert abs(p["area"] - math.pi * a * b) < 0.05 * math.pi * a * b


def test_click_follows_open_closed_config2():
    o = oracle.OracleStream(*synth.shape(2))
    o.learn(synth.learn_frames(2))
    agree = 0
    ts = list(range(0, 120, 3))
    for t in ts:
        _, _, p, _ = o.process(synth.run_frame(2, 0, t))
        agree += p["click"] == (0 if synth.truth(2, 0, t)[1] else 1)
    assert agree >= 0.8 * len(ts)


# --------------------------------------------------------------------------- #
# Re-learning (Sec. 3.3: part of the learning restarted as lighting drifts)   #
# --------------------------------------------------------------------------- #
FIXED_GAIN = dict(gain_min_q16=65536, gain_max_q16=65536)   # c' = c: no brightness term


def test_relearn_windows_are_the_last_frames_of_each_period():
    got = [f for f in range(1, 31) if oracle.relearn_in_window(f, 10, 3)]
    assert got == [8, 9, 10, 18, 19, 20, 28, 29, 30]
    assert not any(oracle.relearn_in_window(f, 10, 0) for f in range(1, 31))
    assert not any(oracle.relearn_in_window(f, 0, 3) for f in range(1, 31))
    assert all(oracle.relearn_in_window(f, 4, 4) for f in range(1, 13))


def _flat(v, h=6, w=8):
    return np.full((h, w, 3), v, np.uint8)


def test_relearned_band_closed_form():
    """Constant background B learned (sigma 0: band [B - d, B + d]); a window of
    R frames at B + 1 (inside the band) re-forms every band to [B + 1 - d, B + 1 + d]:
    S' = R (B + 1), Q' = R (B + 1)^2, n = R gives mu = B + 1, sigma = 0."""
    B, d, R = 100, 2, 3
    o = oracle.OracleStream(8, 6, relearn_frames=R, relearn_min=R, relearn_period=5,
                            bg_margin=d, **FIXED_GAIN)
    o.learn(np.stack([_flat(B)] * 4))
    assert (o.lo == B - d).all() and (o.hi == B + d).all()
    for f in range(1, 6):
        o.process(_flat(B + 1))
        if f < 5:
            assert (o.lo == B - d).all() and (o.hi == B + d).all(), f
    assert (o.lo == B + 1 - d).all() and (o.hi == B + 1 + d).all()
    assert (o.relearn.cnt == 0).all() and (o.relearn.S == 0).all()   # reset after the window


def test_relearn_keeps_bands_of_pixels_seen_as_foreground():
    """A pixel outside its band in the window frames is never counted and keeps
    its band; a pixel counted fewer than relearn_min times keeps it too."""
    B, d = 80, 2
    o = oracle.OracleStream(8, 6, relearn_frames=4, relearn_min=3, relearn_period=4,
                            bg_margin=d, **FIXED_GAIN)
    o.learn(np.stack([_flat(B)] * 3))
    frames = []
    for t in range(4):
        f = _flat(B + 1)
        f[2, 3] = B + 50                        # always outside: count 0
        if t >= 2:
            f[4, 5] = B + 50                    # background in 2 of 4 frames only
        frames.append(f)
    for f in frames:
        o.process(f)
    assert o.lo[2, 3, 0] == B - d and o.hi[2, 3, 0] == B + d
    assert o.lo[4, 5, 0] == B - d and o.hi[4, 5, 0] == B + d
    assert o.lo[0, 0, 0] == B + 1 - d and o.hi[0, 0, 0] == B + 1 + d


def test_relearn_windows_do_not_accumulate_across_windows():
    B, d = 60, 2
    o = oracle.OracleStream(8, 6, relearn_frames=2, relearn_min=2, relearn_period=2,
                            bg_margin=d, **FIXED_GAIN)
    o.learn(np.stack([_flat(B)] * 3))
    for v in (B + 1, B + 1, B + 2, B + 2):
        o.process(_flat(v))
    # second window alone: mu = B + 2, sigma 0
    assert (o.lo == B + 2 - d).all() and (o.hi == B + 2 + d).all()


def test_relearning_tracks_a_drifting_background():
    """The background drifts by +1 level every 2 frames.  Without re-learning
    it leaves the learned band (d = 2) after a few frames and every pixel is
    classified foreground; with a window of 2 every 4 frames the band follows."""
    B, d = 90, 2
    def run(**rl):
        o = oracle.OracleStream(8, 6, bg_margin=d, **FIXED_GAIN, **rl)
        o.learn(np.stack([_flat(B)] * 4))
        outside = []
        for t in range(40):
            f = _flat(B + t // 2)
            outside.append(bool(((f < o.lo) | (f > o.hi)).any()))
            o.process(f)
        return outside
    assert any(run())
    assert not any(run(relearn_frames=2, relearn_min=1, relearn_period=4))


def test_relearning_off_changes_nothing():
    frames = [synth.run_frame(1, 0, t) for t in range(3)]
    lf = synth.learn_frames(1, 0, 8)
    a = oracle.OracleStream(320, 240)
    b = oracle.OracleStream(320, 240, relearn_frames=0, relearn_min=0, relearn_period=50)
    a.learn(lf)
    b.learn(lf)
    for f in frames:
        ra, rb = a.process(f), b.process(f)
        assert np.array_equal(ra[0], rb[0]) and ra[2] == rb[2]


# --------------------------------------------------------------------------- #
# Tracking (Sec. 2: the Mouse module tracks the hand zone)                     #
# --------------------------------------------------------------------------- #
def _two_blobs():
    """A 40x20 label image: blob A (label 0, area 60, 6x10 at x 0..5) and blob
    B (label 30, area 100, 10x10 at x 30..39), found by the oracle's labelling."""
    m = np.zeros((20, 40), np.uint8)
    m[0:10, 0:6] = 1
    m[0:10, 30:40] = 1
    return oracle.label(m)[0]


def test_tracking_picks_the_blob_nearest_the_tracked_point():
    lab = _two_blobs()
    big = oracle.pointer_from_labels(lab, 50)
    assert big["area"] == 100 and big["label"] == 30
    p, tr = oracle.pointer_select(lab, 50, 1000, (1, 3, 4))        # inside A's box
    assert p["area"] == 60 and p["label"] == 0
    # the tracked point moves to A's rounded centroid: sum x = 10 * (0+..+5) = 150,
    # (2*150 + 60) // 120 = 3; sum y = 6 * 45 = 270, (540 + 60) // 120 = 5
    assert tr == (1, 3, 5)
    p, _ = oracle.pointer_select(lab, 50, 1000, (1, 25, 4))       # 20 from A, 5 from B
    assert p["label"] == 30


def test_tracking_falls_back_to_the_largest():
    lab = _two_blobs()
    assert oracle.pointer_select(lab, 50, 1000, (0, 3, 4))[0]["label"] == 30   # no history
    assert oracle.pointer_select(lab, 50, 0, (1, 3, 4))[0]["label"] == 30      # tracking off
    # A's box is x 0..5, y 0..9: point (3, 19) is 10 below it: within 10, beyond 9
    assert oracle.pointer_select(lab, 50, 10, (1, 3, 19))[0]["label"] == 0
    assert oracle.pointer_select(lab, 50, 9, (1, 3, 19))[0]["label"] == 30
    assert oracle.pointer_select(lab, 61, 1000, (1, 3, 4))[0]["label"] == 30   # A below min_area


def test_tracking_ties_prefer_larger_then_smaller_label():
    m = np.zeros((20, 40), np.uint8)
    m[0:10, 0:6] = 1          # label 0, area 60, box x 0..5
    m[0:10, 15:21] = 1        # label 15, area 60, box x 15..20
    m[12:20, 30:40] = 1       # larger, far away
    lab = oracle.label(m)[0]
    p, _ = oracle.pointer_select(lab, 50, 1000, (1, 10, 4))       # 5 from both
    assert p["label"] == 0
    m[0:11, 15:21] = 1        # label 15 now area 66: the larger of the two at distance 5
    p, _ = oracle.pointer_select(oracle.label(m)[0], 50, 1000, (1, 10, 4))
    assert p["label"] == 15


def test_tracking_in_a_stream_follows_the_hand_past_a_larger_distractor():
    """Stream level: a small skin blob moves right while a distractor grows
    larger than it; with tracking the pointer stays on the moving blob."""
    h, w = 48, 96
    bg = np.zeros((h, w, 3), np.uint8)
    bg[..., 2] = 180                                  # blue: never skin
    skin = np.array([200, 140, 110], np.uint8)
    def frame(t):
        f = bg.copy()
        f[10:22, 4 + 2 * t:16 + 2 * t] = skin         # the hand, 12x12, moving
        s = 6 + 2 * t
        f[30:30 + s // 2 + 4, 60:60 + s] = skin       # the distractor, growing
        return f
    common = dict(gain_min_q16=65536, gain_max_q16=65536, min_area=20)
    a = oracle.OracleStream(w, h, **common)
    b = oracle.OracleStream(w, h, track_max_dist=30, **common)
    for o in (a, b):
        o.learn(np.stack([bg] * 3))
    xs_a, xs_b = [], []
    for t in range(12):
        xs_a.append(a.process(frame(t))[2]["x"])
        xs_b.append(b.process(frame(t))[2]["x"])
    assert xs_b == sorted(xs_b) and xs_b[-1] < 40     # stayed on the hand
    assert xs_a[-1] > 60                              # the largest blob is the distractor


# --------------------------------------------------------------------------- #
# Interface module and driving wheel (Sec. 2, Sec. 4)                          #
# --------------------------------------------------------------------------- #
def test_diamond_angle_closed_forms():
    """Axes and diagonals land on exact quarter and eighth turns; the angle
    grows clockwise and is monotone along a circle."""
    assert [oracle.diamond_angle(*d) for d in ((0, -5), (5, 0), (0, 5), (-5, 0))] == [0, 1024, 2048, 3072]
    assert [oracle.diamond_angle(*d) for d in ((3, -3), (3, 3), (-3, 3), (-3, -3))] == [512, 1536, 2560, 3584]
    assert oracle.diamond_angle(0, 0) == 0
    import math
    prev = -1
    for k in range(360):
        t = 2 * math.pi * k / 360
        a = oracle.diamond_angle(round(1000 * math.sin(t)), -round(1000 * math.cos(t)))
        assert a >= prev or (k > 350 and a < 100), (k, a, prev)
        prev = a


def test_interface_zones_and_wheel():
    zones = [(0, 0, 99, 99, 7), (50, 50, 149, 149, 8)]
    wheel = (1, 300, 200, 80, 120, 64)
    ev = oracle.interface_event(True, 60, 60, 0, zones, wheel)
    assert (ev["zone"], ev["event"], ev["on_wheel"]) == (0, 7, 0)   # first listed zone wins
    assert oracle.interface_event(True, 120, 60, 0, zones, wheel)["event"] == 8
    assert oracle.interface_event(False, 60, 60, 1, zones, wheel)["zone"] == -1
    top = oracle.interface_event(True, 300, 100, 1, [], wheel)     # straight up, radius 100
    assert (top["on_wheel"], top["steer"], top["left"], top["right"], top["throttle"]) == (1, 0, 0, 0, 1)
    right = oracle.interface_event(True, 400, 200, 0, [], wheel)
    assert (right["steer"], right["right"], right["left"], right["throttle"]) == (1024, 1, 0, 0)
    left = oracle.interface_event(True, 200, 200, 0, [], wheel)
    assert (left["steer"], left["left"]) == (-1024, 1)
    assert oracle.interface_event(True, 300, 150, 0, [], wheel)["on_wheel"] == 0    # radius 50: inside
    assert oracle.interface_event(True, 300, 50, 0, [], wheel)["on_wheel"] == 0     # radius 150: outside
    small = oracle.interface_event(True, 305, 100, 0, [], wheel)  # 5 px right of the top: 1024*5/105 = 48
    assert (small["steer"], small["right"]) == (48, 0)             # inside the dead zone of 64
    assert oracle.interface_event(True, 310, 100, 0, [], wheel)["right"] == 1   # 1024*10/110 = 93


# --------------------------------------------------------------------------- #
# Gaussian mixture background (Sec. 2 advanced learning; Sec. 3.3 cites Lee's  #
# adaptive mixture learning)                                                   #
# --------------------------------------------------------------------------- #
from fractions import Fraction


def _mix(npx=1, K=3, N=256, T=70, ln=5, ld=2, s0=15, smin=2):
    return oracle.Mixture(npx, K, N, T, ln, ld, s0, smin)


def test_mixture_hand_worked_fixture(golden_dir):
    m = _mix()
    for row in _golden_rows(golden_dir, "mixture_1px.txt"):
        head, W, M, V, C = row.split("|")
        t, x0, x1, x2, fg = map(int, head.split())
        got = m.step(np.array([[x0, x1, x2]], np.uint8))
        assert m.t == t
        assert int(got[0]) == fg, t
        assert m.W[:, 0].tolist() == list(map(int, W.split())), t
        assert m.M[:, :, 0].reshape(-1).tolist() == list(map(int, M.split())), t
        assert m.V[:, 0].tolist() == list(map(int, V.split())), t
        assert m.C[:, 0].tolist() == list(map(int, C.split())), t


def test_mixture_constant_pixel_closed_form():
    """A constant value: one component with the exact mean, full weight and count
    n; its variance follows V0 * prod_{r=2..n} (1 - 1/r) = V0 / n (telescoping),
    each of the n - 1 roundings adding at most 1/2 scaled by r/n: |err| <= (n+1)/4."""
    n, s0 = 40, 15
    m = _mix(npx=2, s0=s0)
    x = np.array([[37, 180, 99], [0, 255, 128]], np.uint8)
    fgs = [m.step(x) for _ in range(n)]
    assert fgs[0].tolist() == [1, 1] and all(f.tolist() == [0, 0] for f in fgs[1:])
    assert (m.M[0] == 256 * x.T.astype(np.uint16)).all()
    assert (m.W[0] == 32768).all() and (m.W[1:] == 0).all()
    assert (m.C[0] == n).all() and (m.C[1:] == 0).all()
    exact = 16 * s0 * s0 / n
    assert (np.abs(m.V[0].astype(float) - exact) <= (n + 1) / 4).all()


def test_mixture_mean_is_the_running_average():
    """With every value matching one component and n <= N, the 1/C rate makes
    the mean the plain average of the values, within (n+1)/4 in Q8 (each step
    rounds by at most 1/2; the error of step i is scaled by i/n)."""
    rng = np.random.default_rng(5)
    m = _mix(npx=64, ln=15, ld=1, s0=63)         # lambda*sigma far above the spread
    vals = rng.integers(100, 141, size=(30, 64, 3), dtype=np.uint8)
    for v in vals:
        m.step(v)
    n = len(vals)
    assert (m.C[0] == n).all() and (m.C[1:] == 0).all()
    for p in range(64):
        for ch in range(3):
            mean = Fraction(int(vals[:, p, ch].astype(int).sum()) * 256, n)
            assert abs(Fraction(int(m.M[0, ch, p])) - mean) <= Fraction(n + 1, 4)


def test_mixture_weights_are_match_frequencies_then_forget_at_rate_1_over_N():
    """Two values that never match each other.  For t <= N the 1/t rate makes
    each weight 32768 * (its frames so far) / t (error <= (t+1)/4); after that,
    frames of B only shrink A's weight by the factor (1 - 1/N) per frame (error
    <= N/2, the rounding geometric sum)."""
    rng = np.random.default_rng(9)
    A, B = np.array([[20, 30, 200]], np.uint8), np.array([[220, 120, 40]], np.uint8)
    N = 64
    m = _mix(N=N)
    seq = rng.random(N) < 0.6
    nA = 0
    for t, isA in enumerate(seq, start=1):
        m.step(A if isA else B)
        nA += int(isA)
        comp = {tuple(m.M[k, :, 0] // 256): int(m.W[k, 0]) for k in range(3) if m.C[k, 0]}
        wA, wB = comp.get((20, 30, 200), 0), comp.get((220, 120, 40), 0)
        assert abs(wA - Fraction(32768 * nA, t)) <= Fraction(t + 1, 4), t
        assert abs(wB - Fraction(32768 * (t - nA), t)) <= Fraction(t + 1, 4), t
    w0 = comp[(20, 30, 200)]
    for s in range(1, 200):
        m.step(B)
        wA = {tuple(m.M[k, :, 0] // 256): int(m.W[k, 0]) for k in range(3) if m.C[k, 0]}.get((20, 30, 200), 0)
        assert abs(wA - w0 * (1 - 1 / N) ** s) <= N / 2, s


def test_mixture_match_radius_is_lambda_sigma():
    """sigma0 = 4, lambda = 5/2: after one frame at x, a value whose mean
    squared channel deviation is lambda^2 sigma^2 = 100 (squared distance 300)
    matches, and one just beyond does not."""
    base = np.array([[100, 100, 100]], np.uint8)
    for off, match in (((10, 10, 10), True), ((10, 10, 11), False), ((17, 0, 0), True),
                       ((18, 0, 0), False), ((0, -10, 14), True), ((1, 10, 14), True),
                       ((2, 10, 14), True), ((3, 10, 14), False), ((-10, -10, -10), True)):
        m = _mix(s0=4)
        m.step(base)
        fg = m.step((base.astype(int) + off).astype(np.uint8))
        assert int((m.C[:, 0] > 0).sum()) == (1 if match else 2), off
        assert int(fg[0]) == (0 if match else 1), off


def test_mixture_background_share_threshold():
    """After A on 60 % and B on 40 % of the frames, A is first in fitness order;
    B is background iff A's share (0.6) is at most T."""
    A, B = np.array([[20, 30, 200]], np.uint8), np.array([[220, 120, 40]], np.uint8)
    for T, b_is_fg in ((70, 0), (50, 1)):
        m = _mix(T=T)
        for t in range(50):
            m.step(A if (t % 5) < 3 else B)
        assert tuple(m.M[0, :, 0] // 256) == (20, 30, 200)
        assert int(m.step(A)[0]) == 0
        assert int(m.step(B)[0]) == b_is_fg, T


def test_mixture_fitness_order_is_kept():
    """After every step: non-empty components first, ordered by W / sqrt(V)."""
    rng = np.random.default_rng(11)
    for K in (2, 3, 4):
        m = _mix(npx=256, K=K, N=16, s0=6)
        for _ in range(40):
            m.step(rng.integers(0, 256, size=(256, 3), dtype=np.uint8) // 64 * 64)
            W, V, C = m.W.astype(object), m.V.astype(object), m.C
            for k in range(K - 1):
                assert not ((C[k] == 0) & (C[k + 1] > 0)).any()
                both = (C[k] > 0) & (C[k + 1] > 0)
                lhs = W[k] * W[k] * V[k + 1]
                rhs = W[k + 1] * W[k + 1] * V[k]
                assert all(l >= r for l, r, b in zip(lhs, rhs, both) if b)


def test_mixture_k1_rate1_is_frame_differencing():
    """K = 1, N = 1: the single component is always the previous frame (matched
    with rate 1 or replaced), with full weight: plain frame differencing."""
    rng = np.random.default_rng(3)
    m = _mix(npx=32, K=1, N=1)
    prev = None
    for _ in range(10):
        x = rng.integers(0, 256, size=(32, 3), dtype=np.uint8)
        fg = m.step(x)
        if prev is None:
            assert (fg == 1).all()
        assert (m.M[0] == 256 * x.T.astype(np.uint16)).all()
        assert (m.W[0] == 32768).all()
        prev = x


def test_mixture_stream_finds_the_generated_hand_config1():
    o = oracle.OracleStream(*synth.shape(1), bg_model=1)
    o.learn(synth.learn_frames(1))
    assert o.mix.t == synth.learn_frames(1).shape[0]
    for t in range(0, 60, 7):
        _, _, p, _ = o.process(synth.run_frame(1, 0, t))
        (cx, cy, a, b), = synth.truth(1, 0, t)[0]
        assert p["valid"] == 1
        assert abs(p["x"] - cx) < 1.0 and abs(p["y"] - cy) < 1.0
        assert abs(p["area"] - math.pi * a * b) < 0.1 * math.pi * a * b


def test_mixture_background_share_boundary_is_inclusive():
    """A then B: both weights 16384, equal fitness, A first.  With T = 50 %,
    B's preceding share is exactly T, which still counts as background."""
    A, B = np.array([[20, 30, 200]], np.uint8), np.array([[220, 120, 40]], np.uint8)
    m = _mix(T=50)
    m.step(A)
    m.step(B)
    assert m.W[:2, 0].tolist() == [16384, 16384]
    assert int(m.step(B)[0]) == 0
    m = _mix(T=49)
    m.step(A)
    m.step(B)
    assert int(m.step(B)[0]) == 1


def test_mixture_first_matching_component_in_fitness_order_is_updated():
    """A = (100,50,50), then B = (180,50,50) (squared distance 6400 > 3 lambda^2
    sigma0^2 = 4218.75: a new component), both with weight 16384 and V0;
    x = (140,50,50) is at 1600 from both, inside both radii: it updates A, the
    first in order (its mean moves half way, rate 1/2), and leaves B alone."""
    m = _mix()
    for v in ((100, 50, 50), (180, 50, 50), (140, 50, 50)):
        m.step(np.array([v], np.uint8))
    assert m.M[0, :, 0].tolist() == [256 * 100 + 5120, 256 * 50, 256 * 50]
    assert m.M[1, :, 0].tolist() == [256 * 180, 256 * 50, 256 * 50]
    assert m.C[:2, 0].tolist() == [2, 1]


def test_mixture_variance_tracks_the_mean_squared_deviation():
    """Values alternating a, a + 12 in one channel (all matching one component).
    With the 1/C rate, V_n = (V0 + sum_{i=2..n} T_i) / n, T_i = 16 (x_i - mean_{i-1})^2 / 3
    per channel (Q4); computed here with exact rational running means.  The
    oracle's roundings stay within (n+1)/4 of V plus what its Q8 means move T."""
    a, d, n = 90, 12, 60
    m = _mix()
    xs = [a + d * (i % 2) for i in range(n)]
    mean, tot = Fraction(xs[0]), Fraction(0)
    for i, x in enumerate(xs):
        m.step(np.array([[x, 50, 50]], np.uint8))
        if i > 0:
            tot += Fraction(16, 3) * (x - mean) ** 2
            mean += (x - mean) / (i + 1)
    exact = (Fraction(3600) + tot) / n
    assert abs(int(m.V[0, 0]) - exact) <= Fraction(n + 1, 4) + 10


def test_mixture_variance_clamps_at_both_ends():
    """A constant value drives V down to exactly Vmin = 16 sigma_min^2 and
    keeps it there; one far value that still matches (lambda 15) pulls V up to
    the 65535 ceiling."""
    m = _mix(s0=15, smin=2)
    x = np.array([[90, 100, 110]], np.uint8)
    for _ in range(200):
        m.step(x)
    assert int(m.V[0, 0]) == 16 * 2 * 2
    m = _mix(ln=15, ld=1, s0=63, smin=1, N=1)
    m.step(np.array([[0, 0, 0]], np.uint8))
    m.step(np.array([[255, 255, 255]], np.uint8))      # D / 3 = 255^2 * 16 > 65535
    assert int(m.C[0, 0]) == 2 and int(m.V[0, 0]) == 65535


def test_mixture_match_count_saturates():
    m = _mix(N=8)
    x = np.array([[10, 200, 30]], np.uint8)
    for _ in range(65540):
        m.step(x, classify=False)
    assert int(m.C[0, 0]) == 65535
    assert int(m.W[0, 0]) == 32768 and (m.M[0, :, 0] == 256 * x[0].astype(np.uint16)).all()


def test_mixture_learning_is_the_update_without_decisions():
    """orc_mixture_learn from an empty model equals stepping the same frames
    one by one (t = 1..n) with no background decisions."""
    rng = np.random.default_rng(21)
    frames = rng.integers(0, 256, size=(9, 5, 7, 3), dtype=np.uint8) // 32 * 32
    a, b = _mix(npx=35, K=4, N=4, s0=9), _mix(npx=35, K=4, N=4, s0=9)
    a.learn(frames)
    for f in frames:
        b.step(f, classify=False)
    assert a.t == b.t == 9
    assert np.array_equal(a.planes(), b.planes())
