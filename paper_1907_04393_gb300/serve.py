"""Replay of camera arrival traces against the continuous-batching server.

The workload: many camera streams of the 256-stream resolution mix, each
sending frames at 30 fps with exponential inter-arrival times, optionally
joining (Poisson arrivals) and leaving (exponential lifetimes) while the trace
runs, with admission limited by the server's device-memory budget (a refused
stream retries every 100 ms).  The trace is replayed in wall-clock time; the
latency of a frame is its completion time minus its scheduled arrival time.

Two ways to serve the same trace are provided: ``run_served`` (the library's
server: resident streams, one tick over every stream with a pending frame) and
``run_plain`` (one synchronous ``hmi_process_frame`` call per frame, in
arrival order, from one worker thread).  This module drives the C ABI only; it
holds none of the method's arithmetic.
"""
from __future__ import annotations

import ctypes
import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import hmi, synth

CFG = 5
FPS = 30.0


@dataclass
class StreamPlan:
    idx: int          # trace-wide stream number
    src: int          # generator stream of configuration 5 (idx mod 256)
    w: int
    h: int
    start: float      # seconds from trace start
    end: float
    arrivals: np.ndarray = field(default_factory=lambda: np.zeros(0))


@dataclass
class Trace:
    duration: float
    streams: list


def make_trace(duration: float, n_streams: int = 256, rate_scale: float = 1.0, churn: bool = True,
               lifetime_mean: float = 20.0, seed: int = 1907043935) -> Trace:
    """All `n_streams` streams start at t = 0; with churn, lifetimes are
    exponential (mean `lifetime_mean` s) and new streams join as a Poisson
    process at n_streams / lifetime_mean per second, so the number of live
    streams stays near n_streams.  Frames arrive per stream as a Poisson
    process at FPS * rate_scale."""
    rng = np.random.default_rng(seed)
    plans = []
    starts = [0.0] * n_streams
    if churn:
        t, rate = 0.0, n_streams / lifetime_mean
        while True:
            t += rng.exponential(1.0 / rate)
            if t >= duration:
                break
            starts.append(t)
    for k, t0 in enumerate(starts):
        src = k % synth.num_streams(CFG)
        w, h = synth.shape(CFG, src)
        end = t0 + rng.exponential(lifetime_mean) if churn else duration
        end = min(end, duration)
        lam = FPS * rate_scale
        gaps = rng.exponential(1.0 / lam, size=int((end - t0) * lam * 1.5) + 16)
        arr = t0 + np.cumsum(gaps)
        plans.append(StreamPlan(k, src, w, h, t0, end, arr[arr < end]))
    return Trace(duration, plans)


class FrameBank:
    """Learning frames and a small ring of run frames per generator stream,
    generated once (pinned host memory, so by-reference submits copy fast)."""

    def __init__(self, srcs, n_learn: int, ring: int = 2):
        import torch
        self.learn, self.ring = {}, {}
        for s in sorted(set(srcs)):
            self.learn[s] = synth.learn_frames(CFG, s, n_learn)
            frames = []
            for t in range(ring):
                f = torch.from_numpy(synth.run_frame(CFG, s, t)).pin_memory()
                frames.append(f)
            self.ring[s] = frames


def _stats(lat_ms, wall_s, nframes, dropped):
    lat = np.sort(np.asarray(lat_ms)) if lat_ms else np.zeros(1)
    return {"frames": int(nframes), "dropped": int(dropped), "wall_s": wall_s,
            "frames_per_s": nframes / wall_s if wall_s > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat[-1])}


def _events(trace: Trace):
    ev = []
    for sp in trace.streams:
        ev.append((sp.start, 0, sp.idx, -1))           # start (admission attempt)
        for n, t in enumerate(sp.arrivals):
            ev.append((float(t), 1, sp.idx, n))        # frame arrival
        ev.append((sp.end, 2, sp.idx, -1))             # end
    heapq.heapify(ev)
    return ev


def run_served(trace: Trace, bank: FrameBank, budget_bytes: int, n_learn: int,
               max_queue: int = 8) -> dict:
    srv = hmi.hmi_server_create(budget_bytes, max_queue)
    plans = {sp.idx: sp for sp in trace.streams}
    sid, arrival = {}, {}
    lat, got = [], [0]
    refused = [0]
    stop = threading.Event()
    buf = (hmi.hmi_server_result * 256)()

    def poller():
        while not stop.is_set() or got[0] < len(arrival):
            n = hmi.hmi_server_poll(srv, buf, 200)
            for k in range(n):
                r = buf[k]
                a = arrival.pop(r.tag, None)
                if a is not None:
                    lat.append((r.done_ns - a) / 1e6)
            if stop.is_set() and not arrival:
                break

    ev = _events(trace)
    pending_retry = []
    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = hmi.hmi_server_now_ns()
    dropped, tag = 0, 0
    while ev or pending_retry:
        if pending_retry and (not ev or pending_retry[0][0] <= ev[0][0]):
            item = heapq.heappop(pending_retry)
        else:
            item = heapq.heappop(ev)
        t, kind, idx, n = item
        delay = t0 + int(t * 1e9) - hmi.hmi_server_now_ns()
        if delay > 0:
            time.sleep(delay / 1e9)
        sp = plans[idx]
        if kind == 0:
            try:
                sid[idx] = hmi.hmi_server_admit(srv, sp.w, sp.h, None, bank.learn[sp.src], n_learn)
            except hmi.HmiError as e:
                if e.status != hmi.HMI_ERR_NO_MEMORY:
                    raise
                refused[0] += 1
                if t + 0.1 < sp.end:
                    heapq.heappush(pending_retry, (t + 0.1, 0, idx, -1))
        elif kind == 1:
            if idx not in sid:
                dropped += 1
                continue
            tag += 1
            arrival[tag] = t0 + int(t * 1e9)
            frame = bank.ring[sp.src][n % len(bank.ring[sp.src])]
            if hmi.hmi_server_submit_ref(srv, sid[idx], frame, tag) != hmi.HMI_OK:
                arrival.pop(tag, None)
                dropped += 1
            else:
                got[0] += 1
        else:
            if idx in sid:
                hmi.hmi_server_release(srv, sid.pop(idx))
    stop.set()
    th.join(timeout=30)
    wall = (hmi.hmi_server_now_ns() - t0) / 1e9
    _, ticks, frames = hmi.hmi_server_stats(srv)
    hmi.hmi_server_destroy(srv)
    out = _stats(lat, wall, len(lat), dropped)
    out.update({"ticks": ticks, "frames_per_tick": frames / max(ticks, 1),
                "admission_refusals": refused[0]})
    return out


def run_plain(trace: Trace, bank: FrameBank, n_learn: int) -> dict:
    """One hmi_process_frame per frame, in arrival order, one worker thread."""
    streams = {}
    for sp in trace.streams:
        s = hmi.Stream(sp.w, sp.h)
        s.learn(bank.learn[sp.src])
        streams[sp.idx] = s
    arr = [(float(t), sp.idx, n) for sp in trace.streams for n, t in enumerate(sp.arrivals)]
    arr.sort()
    lat = []
    ptr = hmi.hmi_pointer()
    t0 = hmi.hmi_server_now_ns()
    for t, idx, n in arr:
        due = t0 + int(t * 1e9)
        delay = due - hmi.hmi_server_now_ns()
        if delay > 0:
            time.sleep(delay / 1e9)
        sp_src = trace.streams[idx].src
        frame = bank.ring[sp_src][n % len(bank.ring[sp_src])]
        hmi.hmi_process_frame(streams[idx].handle, frame, None, ptr)
        lat.append((hmi.hmi_server_now_ns() - due) / 1e6)
    wall = (hmi.hmi_server_now_ns() - t0) / 1e9
    for s in streams.values():
        s.close()
    return _stats(lat, wall, len(lat), 0)
