"""Server: admission by memory budget, per-stream order, and identical results
alone and in the mix (continuous batching does not change any stream's
output)."""
import numpy as np
import pytest

from paper_1907_04393_gb300 import hmi, serve, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_admission_budget_and_refusal():
    one = hmi.hmi_stream_device_bytes(320, 240)
    srv = hmi.hmi_server_create(int(2.5 * one), 4)
    lf = synth.learn_frames(5, 0, 3)
    a = hmi.hmi_server_admit(srv, 320, 240, None, lf, 3)
    b = hmi.hmi_server_admit(srv, 320, 240, None, lf, 3)
    with pytest.raises(hmi.HmiError) as e:
        hmi.hmi_server_admit(srv, 320, 240, None, lf, 3)
    assert e.value.status == hmi.HMI_ERR_NO_MEMORY
    used, _, _ = hmi.hmi_server_stats(srv)
    assert used == 2 * one
    hmi.hmi_server_release(srv, a)
    # the release is applied by the dispatcher; admission succeeds once it has been
    for _ in range(200):
        try:
            hmi.hmi_server_admit(srv, 320, 240, None, lf, 3)
            break
        except hmi.HmiError:
            buf = (hmi.hmi_server_result * 4)()
            hmi.hmi_server_poll(srv, buf, 5000)
    else:
        raise AssertionError("released stream never freed its budget")
    assert b > 0
    hmi.hmi_server_destroy(srv)


def test_served_results_equal_alone_and_in_order():
    """Six streams of mixed sizes, frames submitted interleaved (several per
    stream queued at once): every stream's pointers equal those of the same
    frames processed alone, in the same order."""
    srcs = [0, 1, 130, 140, 200, 245]
    n_learn, nframes = 5, 7
    frames = {s: [synth.run_frame(5, s, t) for t in range(nframes)] for s in srcs}
    learn = {s: synth.learn_frames(5, s, n_learn) for s in srcs}
    alone = {}
    for s in srcs:
        st = hmi.Stream(*synth.shape(5, s))
        st.learn(learn[s])
        alone[s] = [st.process(f, mask=False)[1] for f in frames[s]]
        st.close()
    srv = hmi.hmi_server_create(1 << 34, 16)
    ids = {s: hmi.hmi_server_admit(srv, *synth.shape(5, s), None, learn[s], n_learn) for s in srcs}
    tag_of = {}
    tag = 0
    for t in range(nframes):
        for s in srcs:
            tag += 1
            tag_of[tag] = (s, t)
            assert hmi.hmi_server_submit(srv, ids[s], frames[s][t], tag) == hmi.HMI_OK
    got = {}
    buf = (hmi.hmi_server_result * 64)()
    seen_order = {s: [] for s in srcs}
    while len(got) < tag:
        n = hmi.hmi_server_poll(srv, buf, 2_000_000)
        assert n > 0, "server stalled"
        for k in range(n):
            r = buf[k]
            assert r.status == hmi.HMI_OK
            s, t = tag_of[r.tag]
            got[(s, t)] = r.pointer.as_dict()
            seen_order[s].append(t)
            assert r.done_ns >= r.submit_ns
    for s in srcs:
        assert seen_order[s] == list(range(nframes))
        for t in range(nframes):
            assert got[(s, t)] == alone[s][t], (s, t)
    _, ticks, done = hmi.hmi_server_stats(srv)
    assert done == tag and ticks < tag      # frames were batched
    hmi.hmi_server_destroy(srv)


def test_trace_replay_small():
    tr = serve.make_trace(1.0, n_streams=16, rate_scale=1.0, churn=True, lifetime_mean=2.0)
    bank = serve.FrameBank([sp.src for sp in tr.streams], n_learn=3)
    budget = 12 * hmi.hmi_stream_device_bytes(640, 480)
    out = serve.run_served(tr, bank, budget, 3)
    assert out["frames"] > 0 and out["p99_ms"] < 1000
