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
