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
    """A 1.5 s trace of 16 churning streams under a budget below their demand:
    refusals happen, learning frames come back as such, nothing errs, and the
    plain form serves the same frames."""
    tr = serve.make_trace(1.5, n_streams=16, rate_scale=1.0, churn=True, lifetime_mean=2.0)
    bank = serve.FrameBank([sp.src for sp in tr.streams], learn_ring=3, run_ring=2)
    assert all(sp.w == 320 for sp in tr.streams)
    budget = 10 * hmi.hmi_stream_device_bytes(320, 240)
    out = serve.run_served(tr, bank, budget, 3)
    assert out["errors"] == 0 and out["admission_refusals"] > 0 and out["lost_not_admitted"] > 0
    assert out["frames"] > 0 and 0 < out["learning_frames"] <= 3 * out["streams_admitted"]
    assert out["p99_ms"] < 1000
    pl = serve.run_plain(tr, bank, 3)
    assert pl["errors"] == 0 and pl["frames"] > 0
    pa = serve.run_plain_async(tr, bank, 3, n_cuda_streams=4)
    assert pa["errors"] == 0 and pa["frames"] > 0 and pa["p99_ms"] < 1000


@pytest.mark.parametrize("over", [{}, dict(bg_model=1, mix_k=3)])
def test_online_learning_equals_learned_up_front(over):
    """Streams admitted without learning frames take their first n submitted
    frames as the user-free learning frames (status HMI_LEARNING, empty
    pointer) while another stream is processed in the same ticks; their later
    results equal those of streams learned from the same frames up front
    (with the band, and with the Gaussian mixture learned frame by frame)."""
    srcs = [3, 70, 150, 250]
    n_learn, nframes = 6, 5
    learn = {s: synth.learn_frames(5, s, n_learn) for s in srcs}
    frames = {s: [synth.run_frame(5, s, t) for t in range(nframes)] for s in srcs}
    alone = {}
    for s in srcs:
        st = hmi.Stream(*synth.shape(5, s), **over)
        st.learn(learn[s])
        alone[s] = [st.process(f, mask=False)[1] for f in frames[s]]
        st.close()
    srv = hmi.hmi_server_create(1 << 34, 16)
    busy = srcs[0]            # learned up front, busy while the others learn
    prm = hmi.hmi_default_params(**over)
    ids = {s: hmi.hmi_server_admit(srv, *synth.shape(5, s), prm,
                                   learn[s] if s == busy else None, n_learn) for s in srcs}
    seq = {s: ([] if s == busy else list(learn[s])) + frames[s] for s in srcs}
    tag_of, tag = {}, 0
    for k in range(max(len(v) for v in seq.values())):
        for s in srcs:
            if k < len(seq[s]):
                tag += 1
                tag_of[tag] = (s, k)
                assert hmi.hmi_server_submit(srv, ids[s], np.ascontiguousarray(seq[s][k]), tag) == hmi.HMI_OK
    got = {}
    buf = (hmi.hmi_server_result * 64)()
    while len(got) < tag:
        n = hmi.hmi_server_poll(srv, buf, 2_000_000)
        assert n > 0, "server stalled"
        for i in range(n):
            r = buf[i]
            got[tag_of[r.tag]] = (r.status, r.pointer.as_dict())
    empty = {"valid": 0, "click": 0, "x": -1.0, "y": -1.0, "area": 0,
             "x0": -1, "y0": -1, "x1": -1, "y1": -1, "label": -1}
    for s in srcs:
        skip = 0 if s == busy else n_learn
        for k in range(skip):
            assert got[(s, k)] == (hmi.HMI_LEARNING, empty), (s, k)
        for t in range(nframes):
            st, p = got[(s, skip + t)]
            assert st == hmi.HMI_OK and p == alone[s][t], (s, t)
    hmi.hmi_server_destroy(srv)


@pytest.mark.parametrize("over", [{}, dict(bg_model=1, mix_k=3)])
def test_queued_learning_frames_taken_several_per_round(over):
    """Every frame of two streams is queued before the dispatcher has created
    them, so that each round takes several learning frames of a stream at once
    (summed in layers, one batched launch each; the mixture frame by frame in
    order): the round log shows such a round, and the results equal those of
    streams learned from the same frames up front.  One stream's frames are
    pinned (read in place), the other's copied."""
    srcs = [20, 190]
    n_learn, nframes = 11, 4
    learn = {s: synth.learn_frames(5, s, n_learn) for s in srcs}
    frames = {s: [synth.run_frame(5, s, t) for t in range(nframes)] for s in srcs}
    alone = {}
    for s in srcs:
        st = hmi.Stream(*synth.shape(5, s), **over)
        st.learn(learn[s])
        alone[s] = [st.process(f, mask=False)[1] for f in frames[s]]
        st.close()
    seq = {s: list(learn[s]) + frames[s] for s in srcs}
    pinned = {(s, k): torch.from_numpy(np.ascontiguousarray(seq[s][k])).pin_memory()
              for s in srcs[:1] for k in range(len(seq[s]))}
    srv = hmi.hmi_server_create(1 << 34, 64)
    prm = hmi.hmi_default_params(**over)
    ids = {s: hmi.hmi_server_admit(srv, *synth.shape(5, s), prm, None, n_learn) for s in srcs}
    tag_of, tag = {}, 0
    for s in srcs:
        for k in range(len(seq[s])):
            tag += 1
            tag_of[tag] = (s, k)
            if (s, k) in pinned:
                assert hmi.hmi_server_submit_ref(srv, ids[s], pinned[(s, k)].numpy(), tag) == hmi.HMI_OK
            else:
                assert hmi.hmi_server_submit(srv, ids[s], np.ascontiguousarray(seq[s][k]), tag) == hmi.HMI_OK
    got = _collect(srv, tag_of)
    rec = hmi.hmi_server_rounds(srv)
    hmi.hmi_server_destroy(srv)
    assert int(rec["learning"].max()) > len(srcs), "no round took several learning frames of a stream"
    for s in srcs:
        for k in range(n_learn):
            assert got[(s, k)][0] == hmi.HMI_LEARNING, (s, k)
        for t in range(nframes):
            st, p = got[(s, n_learn + t)]
            assert st == hmi.HMI_OK and p == alone[s][t], (s, t)
    del pinned


def test_online_learning_odd_sizes():
    """Streams whose pixel count is not a multiple of 4 (learning frames summed
    one launch per frame, not in the round's batch) or whose width is not a
    multiple of 16 (frames copied, not read in place by the luma pass), next
    to a regular stream: online learning equals learning up front."""
    rng = np.random.default_rng(77)
    shapes = [(37, 29), (40, 24), (64, 48)]
    n_learn, nframes = 4, 4
    base = {sh: rng.integers(0, 256, size=(sh[1], sh[0], 3)) for sh in shapes}
    learn = {sh: np.clip(base[sh] + rng.integers(-2, 3, size=(n_learn,) + base[sh].shape), 0, 255).astype(np.uint8)
             for sh in shapes}
    frames = {}
    for sh in shapes:
        fr = []
        for t in range(nframes):
            f = np.clip(base[sh] + rng.integers(-2, 3, size=base[sh].shape), 0, 255).astype(np.uint8)
            f[5:15, 5:20] = (200, 120, 90)       # a skin-coloured blob
            fr.append(f)
        frames[sh] = fr
    alone = {}
    for sh in shapes:
        st = hmi.Stream(*sh)
        st.learn(learn[sh])
        alone[sh] = [st.process(f, mask=False)[1] for f in frames[sh]]
        st.close()
    srv = hmi.hmi_server_create(1 << 34, 16)
    ids = {sh: hmi.hmi_server_admit(srv, sh[0], sh[1], None, None, n_learn) for sh in shapes}
    tag_of, tag = {}, 0
    pinned = {}
    for k in range(n_learn + nframes):
        for sh in shapes:
            f = learn[sh][k] if k < n_learn else frames[sh][k - n_learn]
            buf = torch.from_numpy(np.ascontiguousarray(f)).pin_memory()
            pinned[(sh, k)] = buf
            tag += 1
            tag_of[tag] = (sh, k)
            assert hmi.hmi_server_submit(srv, ids[sh], buf.numpy(), tag) == hmi.HMI_OK
    got = {}
    buf = (hmi.hmi_server_result * 64)()
    while len(got) < tag:
        n = hmi.hmi_server_poll(srv, buf, 2_000_000)
        assert n > 0, "server stalled"
        for i in range(n):
            r = buf[i]
            got[tag_of[r.tag]] = (r.status, r.pointer.as_dict())
    for sh in shapes:
        for k in range(n_learn):
            assert got[(sh, k)][0] == hmi.HMI_LEARNING, (sh, k)
        for t in range(nframes):
            st, p = got[(sh, n_learn + t)]
            assert st == hmi.HMI_OK and p == alone[sh][t], (sh, t)
    hmi.hmi_server_destroy(srv)


def _submit_all(srv, ids, seq, pinned=False):
    """Submit seq[s][k] for every stream, interleaved k by k; returns the tag
    map and the buffers that must outlive the results."""
    tag_of, tag, keep = {}, 0, []
    order = [(s, k) for k in range(max(len(v) for v in seq.values())) for s, frs in seq.items() if k < len(frs)]
    # pinned buffers are made before the first submission, so that frames
    # arrive faster than rounds finish and rounds queue up behind each other
    bufs = {sk: torch.from_numpy(np.ascontiguousarray(seq[sk[0]][sk[1]])).pin_memory() for sk in order} \
        if pinned else {}
    keep.extend(bufs.values())
    for s, k in order:
        tag += 1
        tag_of[tag] = (s, k)
        if pinned:
            assert hmi.hmi_server_submit_ref(srv, ids[s], bufs[(s, k)].numpy(), tag) == hmi.HMI_OK
        else:
            assert hmi.hmi_server_submit(srv, ids[s], np.ascontiguousarray(seq[s][k]), tag) == hmi.HMI_OK
    return tag_of, keep


def _collect(srv, tag_of):
    got = {}
    buf = (hmi.hmi_server_result * 256)()
    while len(got) < len(tag_of):
        n = hmi.hmi_server_poll(srv, buf, 2_000_000)
        assert n > 0, "server stalled"
        for i in range(n):
            r = buf[i]
            got[tag_of[r.tag]] = (r.status, r.pointer.as_dict())
    return got


def test_rounds_overlap_on_the_device_results_equal_alone():
    """Frames keep arriving while earlier rounds are still on the GPU: the
    dispatcher issues a round before the previous one is posted (the round log
    shows a round issued before its predecessor was done), and every stream's
    pointers still equal those of the same frames processed alone."""
    srcs = [0, 5, 40, 100, 130, 160, 195, 230, 241, 250]
    n_learn, nframes = 4, 12
    learn = {s: synth.learn_frames(5, s, n_learn) for s in srcs}
    frames = {s: [synth.run_frame(5, s, t) for t in range(nframes)] for s in srcs}
    alone = {}
    for s in srcs:
        st = hmi.Stream(*synth.shape(5, s))
        st.learn(learn[s])
        alone[s] = [st.process(f, mask=False)[1] for f in frames[s]]
        st.close()
    srv = hmi.hmi_server_create(1 << 34, 32)
    ids = {s: hmi.hmi_server_admit(srv, *synth.shape(5, s), None, learn[s], n_learn) for s in srcs}
    tag_of, keep = _submit_all(srv, ids, frames, pinned=True)
    got = _collect(srv, tag_of)
    for s in srcs:
        for t in range(nframes):
            st, p = got[(s, t)]
            assert st == hmi.HMI_OK and p == alone[s][t], (s, t)
    rec = hmi.hmi_server_rounds(srv)
    work = rec[rec["frames"] > 0]
    overlapped = int(np.sum(work["issued_ns"][1:] < work["done_ns"][:-1]))
    assert overlapped > 0, "no round was issued while the previous one was in flight"
    hmi.hmi_server_destroy(srv)
    del keep


def test_config5_streams_against_oracle_through_the_server():
    """Eight streams of the serving workload, two of each resolution, admitted
    with online learning (their first 30 submitted frames are the learning
    frames) and served interleaved: every pointer (area, box, label = smallest
    pixel index, centroid, click state) equals the CPU oracle's for the same
    stream learned from the same 30 frames."""
    import oracle
    srcs = [3, 77, 140, 185, 200, 233, 244, 255]   # 320x240 x2, 640x480 x2, 1280x720 x2, 1920x1080 x2
    n_learn, nframes = 30, 16
    learn = {s: synth.learn_frames(5, s, n_learn) for s in srcs}
    frames = {s: [synth.run_frame(5, s, t) for t in range(nframes)] for s in srcs}
    srv = hmi.hmi_server_create(1 << 34, 64)
    ids = {s: hmi.hmi_server_admit(srv, *synth.shape(5, s), None, None, n_learn) for s in srcs}
    seq = {s: list(learn[s]) + frames[s] for s in srcs}
    tag_of, keep = _submit_all(srv, ids, seq)
    got = _collect(srv, tag_of)
    hmi.hmi_server_destroy(srv)
    sizes = set()
    for s in srcs:
        w, h = synth.shape(5, s)
        sizes.add((w, h))
        o = oracle.OracleStream(w, h)
        o.learn(learn[s])
        for k in range(n_learn):
            assert got[(s, k)][0] == hmi.HMI_LEARNING, (s, k)
        for t in range(nframes):
            _, _, p_o, _ = o.process(frames[s][t], want_labels=False)
            st, p = got[(s, n_learn + t)]
            assert st == hmi.HMI_OK, (s, t)
            for key in ("valid", "click", "area", "x0", "y0", "x1", "y1", "label"):
                assert p[key] == p_o[key], (s, t, key, p[key], p_o[key])
            for key in ("x", "y"):
                assert p[key] == pytest.approx(p_o[key], rel=1e-5, abs=1e-6), (s, t, key)
    assert sizes == {(320, 240), (640, 480), (1280, 720), (1920, 1080)}
    del keep
