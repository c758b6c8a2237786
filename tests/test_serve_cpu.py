"""Host logic of the serving workload (no GPU): the arrival trace's statistics,
the SLO test and the latency summary."""
import numpy as np
import pytest

from paper_1907_04393_gb300 import serve


def test_trace_all_streams_start_at_zero_and_frames_arrive_in_order():
    tr = serve.make_trace(5.0, seed=11)
    starts = [sp.start for sp in tr.streams]
    assert starts[:256] == [0.0] * 256
    assert all(s > 0 for s in starts[256:])
    for sp in tr.streams:
        assert sp.start <= sp.end <= 5.0
        a = np.asarray(sp.arrivals)
        assert (np.diff(a) > 0).all() and (a >= sp.start).all() and (a < sp.end).all()
    at, ai, an = serve._arrivals(tr)
    assert at == sorted(at) and len(at) == tr.frames


@pytest.mark.parametrize("scale", [1.0, 4.0])
def test_trace_frame_rate_per_stream(scale):
    """Poisson arrivals at 30 fps x scale: frames / live stream-seconds within
    a few percent (thousands of arrivals)."""
    tr = serve.make_trace(10.0, rate_scale=scale, seed=5)
    live = sum(sp.end - sp.start for sp in tr.streams)
    rate = tr.frames / live
    assert abs(rate - serve.FPS * scale) < 0.03 * serve.FPS * scale


def test_trace_churn_keeps_about_n_streams_live():
    """Joins at n / lifetime per second and exponential lifetimes keep the
    time-averaged number of live streams near n (Little's law)."""
    tr = serve.make_trace(60.0, seed=7)
    ts = np.linspace(1.0, 59.0, 300)
    live = [sum(1 for sp in tr.streams if sp.start <= t < sp.end) for t in ts]
    assert 0.85 * 256 < np.mean(live) < 1.15 * 256
    joins = sum(1 for sp in tr.streams if sp.start > 0)
    assert abs(joins / 60.0 - 256 / 20.0) < 0.2 * 256 / 20.0
    # exponential lifetimes censored at the trace end: the maximum-likelihood
    # mean is the total exposure over the number of streams that ended
    exposure = sum(sp.end - sp.start for sp in tr.streams)
    ended = sum(1 for sp in tr.streams if sp.end < 60.0)
    assert 17.0 < exposure / ended < 23.0


def test_trace_without_churn_and_seed():
    a = serve.make_trace(2.0, churn=False, seed=3)
    b = serve.make_trace(2.0, churn=False, seed=3)
    assert len(a.streams) == 256 and all(sp.end == 2.0 for sp in a.streams)
    assert a.frames == b.frames
    assert all(np.array_equal(x.arrivals, y.arrivals) for x, y in zip(a.streams, b.streams))


def _row(**over):
    r = {"offered_frames_per_s": 1000.0, "wall_s": 5.0, "p99_ms": 1.0, "errors": 0,
         "dropped_queue_full": 0}
    r.update(over)
    return r


def test_slo_boundaries():
    assert serve.meets_slo(_row())
    assert serve.meets_slo(_row(p99_ms=serve.SLO_MS))
    assert not serve.meets_slo(_row(p99_ms=serve.SLO_MS + 1e-9))
    assert serve.meets_slo(_row(dropped_queue_full=int(serve.DROP_BUDGET * 5000)))
    assert not serve.meets_slo(_row(dropped_queue_full=int(serve.DROP_BUDGET * 5000) + 1))
    assert not serve.meets_slo(_row(errors=1))
    assert not serve.meets_slo(_row(saturated=True))


def test_latency_summary():
    lat = list(np.arange(1, 101, dtype=float))
    st = serve._latency_stats(lat)
    assert st["p50_ms"] == pytest.approx(50.5)
    assert st["p99_ms"] == pytest.approx(99.01)
    assert st["max_ms"] == 100.0
    assert serve._latency_stats([])["max_ms"] == 0.0
