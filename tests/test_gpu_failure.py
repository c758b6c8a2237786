"""Failure detection on the GPU without any fault.

Every device-side retry loop and wait is bounded; a loop that runs out sets
the stream's error flag, lets the tick end, and the next synchronous call
returns HMI_ERR_DEVICE_TIMEOUT.  Lowering the batch's bound to one step makes
the component merge of a hand that spans several 32x32 blocks run out (path
lengths of its union-find exceed one step) on both forms of the tick; with the
default bound back, the same stream matches the oracle again.
"""
import numpy as np
import pytest

import oracle
from paper_1907_04393_gb300 import hmi, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ptr_dict(ptrs, i=0):
    return dict(zip(ptrs.dtype.names, [x.item() for x in ptrs[i]]))


@pytest.mark.parametrize("fused", [1, 0, 2])
def test_loop_bound_runs_out_then_stream_recovers(fused):
    w, h = synth.shape(1)
    lf = synth.learn_frames(1)
    g = hmi.Stream(w, h)
    g.learn(torch.from_numpy(lf).cuda())
    b = hmi.hmi_batch_create([g.handle])
    try:
        hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), fused=fused))
        frame = synth.run_frame(1, 0, 5)
        masks = [np.empty((h, w), np.uint8)]
        ptrs = np.zeros(1, hmi.POINTER_DTYPE)
        # the hand at this frame spans several blocks: its merge needs more than one step
        o = oracle.OracleStream(w, h)
        o.learn(lf)
        _, l_o, p_o, _ = o.process(frame)
        assert len({(y // 32, x // 32) for y, x in np.argwhere(l_o == p_o["label"])}) >= 4
        hmi.hmi_batch_set_loop_limit(b, 1)
        with pytest.raises(hmi.HmiError) as e:
            hmi.hmi_batch_process(b, [frame], masks, ptrs)
        assert e.value.status == hmi.HMI_ERR_DEVICE_TIMEOUT
        # the error was reported once; the stream works again with the default bound
        hmi.hmi_batch_set_loop_limit(b, 0)
        hmi.hmi_batch_process(b, [synth.run_frame(1, 0, 6)], masks, ptrs)
        g.learn(torch.from_numpy(lf).cuda())         # fresh click state on both sides
        o = oracle.OracleStream(w, h)
        o.learn(lf)
        for t in (5, 6, 7):
            frame = synth.run_frame(1, 0, t)
            hmi.hmi_batch_process(b, [frame], masks, ptrs)
            m_o, l_o, p_o, _ = o.process(frame)
            assert np.array_equal(masks[0], m_o), f"frame {t} mask"
            assert np.array_equal(g.labels(), l_o), f"frame {t} labels"
            p = _ptr_dict(ptrs)
            for k in ("valid", "click", "area", "x0", "y0", "x1", "y1", "label"):
                assert p[k] == p_o[k], (t, k)
    finally:
        hmi.hmi_batch_destroy(b)
        g.close()
