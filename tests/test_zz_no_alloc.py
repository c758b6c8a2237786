"""The allocation-free gain entry point, checked against the per-frame path.

hmi_frame_gain_noalloc serves callers that cannot allocate device memory (a
real-time loop where cudaMalloc could stall the device, or a host program that
owns all device memory through its own pool).  It must give exactly the gain
that hmi_process_frame applies to the same frame.  This file is collected last
so that a failure here comes after every other test has run; it also passes
when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1907_04393_gb300 import hmi, synth

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_gain_matches_per_frame_path_twice():
    w, h = synth.shape(1)
    st = hmi.Stream(w, h)
    st.learn(torch.from_numpy(synth.learn_frames(1)).cuda())
    syref, _ = hmi.hmi_export_background(st.handle)
    p = st.params
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for t in (5, 29):                      # two calls in a row
        frame = torch.from_numpy(synth.run_frame(1, 0, t)).cuda()
        st.process(frame)
        expect = st.last_gain()
        hmi.hmi_frame_gain_noalloc(frame, w, h, syref, p.gain_min_q16, p.gain_max_q16,
                                   out, stream)
        torch.cuda.synchronize()
        assert int(out.item()) == expect, f"frame {t}"
    st.close()


@pytest.mark.gpu
def test_noalloc_gain_unaligned_width_and_size_limit():
    w, h = 100, 37                         # rows not 16-pixel aligned: scalar reads
    rng = np.random.default_rng(7)
    learn = rng.integers(0, 256, size=(3, h, w, 3), dtype=np.uint8)
    st = hmi.Stream(w, h)
    st.learn(learn)
    syref, _ = hmi.hmi_export_background(st.handle)
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(2):
        frame = torch.from_numpy(rng.integers(0, 256, size=(h, w, 3), dtype=np.uint8)).cuda()
        st.process(frame)
        hmi.hmi_frame_gain_noalloc(frame, w, h, syref, st.params.gain_min_q16,
                                   st.params.gain_max_q16, out, stream)
        torch.cuda.synchronize()
        assert int(out.item()) == st.last_gain()
    with pytest.raises(hmi.HmiError) as e:
        hmi.hmi_frame_gain_noalloc(frame, 8193, 8, syref, 0, 65536, out, stream)
    assert e.value.status == hmi.HMI_ERR_INVALID_ARG
    st.close()


@pytest.mark.gpu
def test_noalloc_gain_full_hd_frame_many_ctas():
    """A 1920x1080 frame spreads over 127 CTAs: the last CTA adds all their
    partial sums; checked against the per-frame path twice in a row."""
    w, h = synth.shape(3)
    st = hmi.Stream(w, h)
    st.learn(torch.from_numpy(synth.learn_frames(3)).cuda())
    syref, _ = hmi.hmi_export_background(st.handle)
    p = st.params
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for t in (0, 17):
        frame = torch.from_numpy(synth.run_frame(3, 0, t)).cuda()
        st.process(frame)
        hmi.hmi_frame_gain_noalloc(frame, w, h, syref, p.gain_min_q16, p.gain_max_q16, out, stream)
        torch.cuda.synchronize()
        assert int(out.item()) == st.last_gain(), f"frame {t}"
    st.close()


@pytest.mark.gpu
def test_noalloc_gain_largest_frame_against_host_luma_sum():
    """The largest accepted frame, 8192 x 8192 (all 4096 scratch slots), against
    the gain of its luma sum computed on the host by the oracle."""
    import oracle
    w = h = 8192
    rng = np.random.default_rng(11)
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for syref_per_px in (90, 160):          # one gain below 1, one above
        host = rng.integers(0, 256, size=(h, w, 3), dtype=np.uint8)
        syref = syref_per_px * w * h
        expect = oracle.gain(oracle.luma_sum(host), syref, 32768, 131072)
        frame = torch.from_numpy(host).cuda()
        hmi.hmi_frame_gain_noalloc(frame, w, h, syref, 32768, 131072, out, stream)
        torch.cuda.synchronize()
        assert int(out.item()) == expect
        del frame


@pytest.mark.gpu
def test_noalloc_gain_rejects_unreachable_buffers_without_running():
    """Buffers a kernel could not use, and an impossible reference luma, are
    refused before any work is enqueued (the output keeps its sentinel) and the
    status is recorded for hmi_last_error."""
    w, h = 64, 8
    frame = torch.zeros((h, w, 3), dtype=torch.uint8, device="cuda")
    out = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pageable = np.zeros((h, w, 3), np.uint8)
    host_out = np.zeros(1, np.uint32)
    cases = [
        (pageable, out.data_ptr(), 100 * w * h),              # pageable host frame
        (frame, host_out, 100 * w * h),                       # gain in host memory
        (frame, out.data_ptr() + 2, 100 * w * h),             # gain not 4-byte aligned
        (frame, out.data_ptr(), 255 * w * h + 1),             # syref beyond any frame's sum
    ]
    for f, g, syref in cases:
        with pytest.raises(hmi.HmiError) as e:
            hmi.hmi_frame_gain_noalloc(f, w, h, syref, 32768, 131072, g, stream)
        assert e.value.status == hmi.HMI_ERR_INVALID_ARG
        assert hmi.hmi_last_error() == hmi.HMI_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert out.tolist() == [-7, -7, -7, -7]
    # pinned host frames are readable by the kernel and accepted
    pinned = torch.zeros((h, w, 3), dtype=torch.uint8).pin_memory()
    hmi.hmi_frame_gain_noalloc(pinned, w, h, 0, 32768, 131072, out, stream)
    torch.cuda.synchronize()
    assert int(out[0].item()) == 65536      # a black frame keeps unit gain before the clamp
