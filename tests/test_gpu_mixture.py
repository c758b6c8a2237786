"""Parity of the Gaussian mixture background (bg_model 1; Sec. 2 advanced
learning of the background, Sec. 3.3 Lee's adaptive mixture) against the CPU
oracle, through the C ABI.

Bar: the whole mixture state (weights, means, variances, counts, in fitness
order) bit-exact after learning and after every checked frame; masks, labels,
blob area and box bit-exact; centroid within 1e-5 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1907_04393_gb300 import hmi, synth
from test_gpu_parity import _dev, assert_pointer, check_frame, pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check_mix(g: hmi.Stream, o: oracle.OracleStream, what=""):
    a, b = g.mixture(), o.mix.planes()
    if not np.array_equal(a, b):
        bad = np.argwhere(a != b)
        raise AssertionError(f"{what} mixture differs at {len(bad)} entries (plane, px), "
                             f"first {bad[:4].tolist()}")


def _frames(w, h, n, seed):
    """Learning-like frames: a fixed random background with small noise."""
    rng = np.random.default_rng(seed)
    base = rng.integers(0, 256, size=(h, w, 3))
    noise = rng.integers(-3, 4, size=(n, h, w, 3))
    return np.clip(base + noise, 0, 255).astype(np.uint8)


@pytest.mark.parametrize("w,h,n,K,dev", [(320, 240, 30, 3, False), (37, 29, 5, 1, True),
                                          (1, 1, 3, 2, False), (33, 65, 17, 4, True),
                                          (312, 40, 12, 3, False)])
def test_mixture_learning_matches_oracle(w, h, n, K, dev):
    g, o = pair(w, h, bg_model=1, mix_k=K)
    lf = _frames(w, h, n, seed=w * 31 + h)
    g.learn(_dev(lf) if dev else lf)
    o.learn(lf)
    _check_mix(g, o, f"{w}x{h} K{K}")
    g.close()


@pytest.mark.parametrize("cfg,K,w_over,over", [(1, 3, None, {}), (2, 2, None, dict(mix_rate_n=16)),
                                               (1, 4, 312, dict(mix_bg_pct=50)),
                                               (1, 1, None, dict(mix_rate_n=1, mix_sigma0=8))])
def test_mixture_frames_match_oracle(cfg, K, w_over, over):
    """Every frame's mask, labels, gain and pointer, and the mixture after
    every frame, equal the oracle's (config 1 and 2 frames; a width that is not
    a multiple of 16; K from 1, the frame-differencing special case, to 4)."""
    w, h = synth.shape(cfg)
    if w_over:
        w = w_over
    g, o = pair(w, h, bg_model=1, mix_k=K, **over)
    lf = np.ascontiguousarray(synth.learn_frames(cfg, 0, 10)[:, :, :w])
    g.learn(lf)
    o.learn(lf)
    _check_mix(g, o, "learned")
    for t in range(14):
        f = np.ascontiguousarray(synth.run_frame(cfg, 0, t)[:, :w])
        check_frame(g, o, f, dev=t % 2 == 1, what=f"cfg{cfg} K{K} w{w} t={t}")
        if t % 3 == 0 or t == 13:
            _check_mix(g, o, f"cfg{cfg} K{K} w{w} t={t}")
    g.close()


def test_mixture_small_and_ragged_sizes():
    for w, h in ((1, 1), (17, 5), (50, 1), (33, 33)):
        g, o = pair(w, h, bg_model=1, mix_k=2, mix_rate_n=4)
        lf = _frames(w, h, 4, seed=w + 100 * h)
        g.learn(lf)
        o.learn(lf)
        rng = np.random.default_rng(w * h)
        for t in range(5):
            f = rng.integers(0, 256, size=(h, w, 3), dtype=np.uint8)
            check_frame(g, o, f, what=f"{w}x{h} t={t}")
        _check_mix(g, o, f"{w}x{h}")
        g.close()


def test_mixture_in_batches_and_pipelines():
    """A batch of band streams, a re-learning stream and mixture streams with
    1, 3 and 4 components: plain graph ticks and pipelined ticks at depths 2
    and 3 match the oracle frame by frame, final mixtures included."""
    idx = [0, 20, 33, 50, 61]
    kinds = [dict(bg_model=1, mix_k=3), {}, dict(bg_model=1, mix_k=1, mix_rate_n=8),
             dict(relearn_frames=3, relearn_min=2, relearn_period=5), dict(bg_model=1, mix_k=4)]
    for mode in ("plain", 2, 3):
        gs, os_ = [], []
        for i, over in zip(idx, kinds):
            w, h = synth.shape(4, i)
            g, o = pair(w, h, **over)
            lf = synth.learn_frames(4, i, 8)
            g.learn(_dev(lf))
            o.learn(lf)
            gs.append(g)
            os_.append(o)
        b = hmi.hmi_batch_create([g.handle for g in gs])
        hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), groups=1,
                                         pipeline_depth=mode if mode != "plain" else 2))
        s = torch.cuda.current_stream().cuda_stream
        T = 10
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
                assert_pointer(dict(zip(arr.dtype.names, [x.item() for x in arr[k]])), p_o,
                               f"{mode} t={t} s={k}")
        for k in range(len(idx)):
            if kinds[k].get("bg_model"):
                _check_mix(gs[k], os_[k], f"{mode} s={k}")
        hmi.hmi_batch_destroy(b)
        for g in gs:
            g.close()


def test_autotune_keeps_adaptive_state():
    """Autotuning between ticks restores the mixtures and the re-learning state
    as well as the click state: later results and final mixtures are those of
    an untuned twin batch."""
    idx = [2, 17, 35, 60]
    kinds = [dict(bg_model=1, mix_k=3), dict(relearn_frames=2, relearn_min=1, relearn_period=3),
             dict(bg_model=1, mix_k=2), {}]
    T = 6
    frames = [[_dev(synth.run_frame(4, i, t)) for i in idx] for t in range(T + 1)]

    def streams():
        out = []
        for i, over in zip(idx, kinds):
            g = hmi.Stream(*synth.shape(4, i), **over)
            g.learn(_dev(synth.learn_frames(4, i, 6)))
            out.append(g)
        return out

    ga, gb = streams(), streams()
    ba = hmi.hmi_batch_create([g.handle for g in ga])
    bb = hmi.hmi_batch_create([g.handle for g in gb])
    s = torch.cuda.current_stream().cuda_stream
    out = {}
    for name, b in (("a", ba), ("b", bb)):
        res = []
        for t in range(T):
            if name == "b" and t == 3:
                hmi.hmi_batch_autotune(b, frames[T], 4, t % 2 == 0)
            p = torch.zeros(len(idx) * 40, dtype=torch.uint8, device="cuda")
            hmi.hmi_batch_process_async(b, frames[t], None, p.data_ptr(), s, False)
            res.append(p)
        torch.cuda.synchronize()
        out[name] = [r.cpu().numpy().view(hmi.POINTER_DTYPE) for r in res]
    for t in range(T):
        assert np.array_equal(out["a"][t], out["b"][t]), t
    for k, over in enumerate(kinds):
        if over.get("bg_model"):
            assert np.array_equal(ga[k].mixture(), gb[k].mixture()), k
        else:
            assert all(np.array_equal(x, y) for x, y in zip(ga[k].band(), gb[k].band())), k
    for b in (ba, bb):
        hmi.hmi_batch_destroy(b)
    for g in ga + gb:
        g.close()


def test_mixture_api_errors():
    band = hmi.Stream(32, 16)
    mix = hmi.Stream(32, 16, bg_model=1)
    with pytest.raises(hmi.HmiError) as e:
        mix.mixture()
    assert e.value.status == hmi.HMI_ERR_NOT_LEARNED
    lf = _frames(32, 16, 3, seed=1)
    band.learn(lf)
    mix.learn(lf)
    out = np.empty((18, 32 * 16), np.uint16)
    with pytest.raises(hmi.HmiError) as e:
        hmi.hmi_get_mixture(band.handle, out)
    assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    z32 = np.zeros((16, 32, 3), np.uint32)
    z8 = np.zeros((16, 32, 3), np.uint8)
    with pytest.raises(hmi.HmiError) as e:
        mix.import_background(z32, z32, z8, z8, 1, 0)
    assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    band.close()
    mix.close()


def test_mixture_full_hd_stream():
    """The third configuration's 1920x1080 stream (two hands, drift, flicker)
    with the mixture: learning from its 30 frames and two running frames give
    the oracle's whole mixture state, masks, labels and pointers."""
    w, h = synth.shape(3)
    g, o = pair(w, h, bg_model=1, mix_k=3)
    lf = synth.learn_frames(3)
    g.learn(_dev(lf))
    o.learn(lf)
    _check_mix(g, o, "1080p learned")
    for t in (0, 1):
        check_frame(g, o, synth.run_frame(3, 0, t), dev=t == 1, what=f"1080p t={t}")
    _check_mix(g, o, "1080p after 2 frames")
    g.close()


def test_mixture_extremes():
    """Counts saturate (65535 learning frames), variances reach both clamps
    (a constant pixel decays to Vmin; a far value that still matches with
    lambda 15 and sigma0 63 clamps at 65535): the GPU state equals the oracle's."""
    rng = np.random.default_rng(8)
    w, h, n = 8, 8, 65535
    base = rng.integers(0, 51, size=(1, h, w, 3), dtype=np.uint8)
    lf = np.repeat(base, n, axis=0)
    # rows 0-3 end with a far value F (a new component, V0) and then F - 100,
    # which only that component matches: its variance jumps to the ceiling;
    # rows 4-7 stay constant: their count saturates, their variance is Vmin
    lf[-2, :4] = 255 - base[0, :4]
    lf[-1, :4] = 155 - base[0, :4]
    over = dict(bg_model=1, mix_k=2, mix_rate_n=1, bg_k_num=15, bg_k_den=1, mix_sigma0=63,
                mix_sigma_min=1)
    g, o = pair(w, h, **over)
    g.learn(lf)
    o.learn(lf)
    _check_mix(g, o, "extremes learned")
    planes = o.mix.planes()
    assert planes[5 * 2:].max() == 65535                # some count saturated
    assert planes[4 * 2:5 * 2].max() == 65535           # some variance at the ceiling
    for t in range(3):
        f = np.ascontiguousarray(base[0] if t % 2 == 0 else 255 - base[0])
        check_frame(g, o, f, what=f"extremes t={t}")
    _check_mix(g, o, "extremes after 3 frames")
    g.close()
