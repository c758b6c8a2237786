"""Replay of camera arrival traces against the continuous-batching server.

The workload: camera streams of the 256-stream resolution mix (128 at
320x240, 64 at 640x480, 48 at 1280x720, 16 at 1920x1080), each sending frames
at 30 fps with exponential inter-arrival times, joining (Poisson arrivals) and
leaving (exponential lifetimes) while the trace runs, with admission limited
by the server's device-memory budget (a refused stream retries every 100 ms,
and its frames are lost until it is admitted).  A stream's first n_learn
frames are its user-free learning frames (Sec. 2: the background is learned
with no hand in view); the server accumulates them online as they arrive.  The
trace is replayed in wall-clock time; the latency of a frame is its completion
time minus its scheduled arrival time, so a submitter running late counts
against the server, never for it.

Two ways to serve the same trace:
  * ``run_served``: the library's server (resident streams, one tick over
    every stream with a pending frame, online learning);
  * ``run_plain``: one synchronous ``hmi_process_frame`` call per frame, in
    arrival order, from one worker thread, with every stream created and
    learned before the trace starts (its learning frames are skipped, so the
    plain form does no learning work while it is timed);
  * ``run_plain_async``: the same per-stream calls made asynchronous: each
    frame is copied to its stream's device buffer and processed by
    ``hmi_process_frame_async`` on one of several CUDA streams, its pointer
    read back, and a completion thread takes the latency when the frame's
    event has passed, so that the frames of different streams overlap on
    the device.

Frames come from a bank of pinned host buffers per generator stream: a ring of
``LEARN_RING`` distinct learning frames, cycled through the n_learn learning
frames, and a ring of run frames.  This module drives the C ABI only; it holds
none of the method's arithmetic.
"""
from __future__ import annotations

import contextlib
import ctypes
import gc
import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import hmi, synth

CFG = 5
FPS = 30.0
N_LEARN = 30
LEARN_RING = 8
RETRY_S = 0.1
SLO_MS = 5.0


@dataclass
class StreamPlan:
    idx: int          # trace-wide stream number
    src: int          # generator stream of the 256-stream mix (idx mod 256)
    w: int
    h: int
    start: float      # seconds from trace start
    end: float
    arrivals: np.ndarray = field(default_factory=lambda: np.zeros(0))


@dataclass
class Trace:
    duration: float
    streams: list

    @property
    def frames(self) -> int:
        return int(sum(len(sp.arrivals) for sp in self.streams))


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
    """Pinned host frames per generator stream: LEARN_RING learning frames and
    `run_ring` run frames, generated once."""

    def __init__(self, srcs, learn_ring: int = LEARN_RING, run_ring: int = 2):
        import torch
        self.learn, self.run, self.addr = {}, {}, {}
        for s in sorted(set(srcs)):
            lf = synth.learn_frames(CFG, s, learn_ring)
            self.learn[s] = [torch.from_numpy(np.ascontiguousarray(f)).pin_memory() for f in lf]
            self.run[s] = [torch.from_numpy(synth.run_frame(CFG, s, t)).pin_memory()
                           for t in range(run_ring)]
            self.addr[s] = ([f.data_ptr() for f in self.learn[s]], [f.data_ptr() for f in self.run[s]])

    def frame_addr(self, src: int, k: int, n_learn: int) -> int:
        """Address of the k-th frame a stream of generator stream `src` sends."""
        la, ra = self.addr[src]
        return la[k % len(la)] if k < n_learn else ra[(k - n_learn) % len(ra)]

    def learn_block(self, src: int, n_learn: int) -> np.ndarray:
        """The n_learn learning frames, contiguous (for up-front learning)."""
        ring = self.learn[src]
        return np.stack([ring[k % len(ring)].numpy() for k in range(n_learn)])


RESULT_DTYPE = np.dtype([("stream_id", np.int32), ("status", np.int32), ("tag", np.uint64),
                         ("submit_ns", np.uint64), ("done_ns", np.uint64),
                         ("pointer", hmi.POINTER_DTYPE)])
assert RESULT_DTYPE.itemsize == ctypes.sizeof(hmi.hmi_server_result)


@contextlib.contextmanager
def _no_gc_pauses():
    """The replay is a load generator: a cyclic-GC pass over the interpreter's
    objects would stall it for tens of ms and show up as server latency."""
    gc.collect()
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def _latency_stats(lat_ms) -> dict:
    lat = np.sort(np.asarray(lat_ms, dtype=np.float64)) if len(lat_ms) else np.zeros(1)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat[-1])}


def _arrivals(trace: Trace):
    """All frame arrivals sorted by time: (t, stream idx, frame number)."""
    t = np.concatenate([sp.arrivals for sp in trace.streams] + [np.zeros(0)])
    idx = np.concatenate([np.full(len(sp.arrivals), sp.idx) for sp in trace.streams] + [np.zeros(0, int)])
    num = np.concatenate([np.arange(len(sp.arrivals)) for sp in trace.streams] + [np.zeros(0, int)])
    o = np.argsort(t, kind="stable")
    return t[o].tolist(), idx[o].astype(int).tolist(), num[o].astype(int).tolist()


def run_served(trace: Trace, bank: FrameBank, budget_bytes: int, n_learn: int = N_LEARN,
               max_queue: int = 8) -> dict:
    with _no_gc_pauses():
        return _run_served(trace, bank, budget_bytes, n_learn, max_queue)


def _run_served(trace: Trace, bank: FrameBank, budget_bytes: int, n_learn: int,
                max_queue: int) -> dict:
    lib = hmi.load()
    srv = hmi.hmi_server_create(budget_bytes, max_queue)
    plans = {sp.idx: sp for sp in trace.streams}
    sid = {}
    arrival = {}                    # tag -> scheduled arrival (ns), outstanding
    lat, lat_at, counts = [], [], {"learn": 0, "errors": 0}
    stop = threading.Event()
    buf = (hmi.hmi_server_result * 1024)()
    view = np.frombuffer(buf, dtype=RESULT_DTYPE)

    def poller():
        deadline = None
        while True:
            n = lib.hmi_server_poll(srv, buf, len(buf), 2000)
            if n > 0:
                for tg, st, dn in zip(view["tag"][:n].tolist(), view["status"][:n].tolist(),
                                      view["done_ns"][:n].tolist()):
                    a = arrival.pop(tg, None)
                    if a is None:
                        continue
                    if st == hmi.HMI_OK:
                        lat.append((dn - a) * 1e-6)
                        lat_at.append(a)
                    elif st == hmi.HMI_LEARNING:
                        counts["learn"] += 1
                    else:
                        counts["errors"] += 1
            if stop.is_set():
                if not arrival:
                    break
                deadline = deadline or time.monotonic() + 30.0
                if time.monotonic() > deadline:
                    break

    # stream starts / ends and retries, merged with the sorted frame arrivals
    ctl = []
    for sp in trace.streams:
        ctl.append((sp.start, 0, sp.idx))
        ctl.append((sp.end, 2, sp.idx))
    heapq.heapify(ctl)
    at, ai, _ = _arrivals(trace)
    th = threading.Thread(target=poller, daemon=True)
    th.start()
    now = lib.hmi_server_now_ns
    submit = lib.hmi_server_submit_ref
    refused = lost = dropped = admitted = 0
    drop_t, lag = [], []
    sent = {}                       # frames each admitted stream has been sent
    tag, j, na = 0, 0, len(at)
    t0 = now()
    while j < na or ctl:
        if ctl and (j >= na or ctl[0][0] <= at[j]):
            t, kind, idx = heapq.heappop(ctl)
        else:
            t, kind, idx = at[j], 1, ai[j]
            j += 1
        due = t0 + int(t * 1e9)
        delay = due - now()
        if delay > 150_000:
            time.sleep((delay - 100_000) * 1e-9)
        if kind == 1:
            s = sid.get(idx)
            if s is None:
                lost += 1                     # stream not (yet) admitted
                continue
            k = sent[idx]
            sent[idx] = k + 1
            tag += 1
            arrival[tag] = due
            lag.append(now() - due)
            if submit(srv, s, bank.frame_addr(plans[idx].src, k, n_learn), tag) != hmi.HMI_OK:
                arrival.pop(tag, None)
                dropped += 1                  # the stream's queue is full
                drop_t.append(t)
        elif kind == 0:
            sp = plans[idx]
            try:
                sid[idx] = hmi.hmi_server_admit(srv, sp.w, sp.h, None, None, n_learn)
                sent[idx] = 0                 # the camera's first frames are user-free
                admitted += 1
            except hmi.HmiError as e:
                if e.status != hmi.HMI_ERR_NO_MEMORY:
                    raise
                refused += 1
                if t + RETRY_S < sp.end:
                    heapq.heappush(ctl, (t + RETRY_S, 0, idx))
        elif idx in sid:
            hmi.hmi_server_release(srv, sid.pop(idx))
    t_end = now()
    stop.set()
    th.join(timeout=60)
    wall = (t_end - t0) * 1e-9
    _, ticks, frames = hmi.hmi_server_stats(srv)
    rounds = hmi.hmi_server_rounds(srv)
    hmi.hmi_server_destroy(srv)
    out = {"frames": len(lat), "frames_per_s": len(lat) / wall, "wall_s": wall,
           "learning_frames": counts["learn"], "errors": counts["errors"],
           "dropped_queue_full": dropped, "lost_not_admitted": lost,
           "streams_admitted": admitted, "admission_refusals": refused,
           "ticks": ticks, "frames_per_tick": frames / max(ticks, 1),
           "offered_frames_per_s": trace.frames / trace.duration}
    out.update(_latency_stats(lat))
    # the start (all streams admitted and learning at once) against the rest
    warm = t0 + int(1e9)
    steady = [x for x, a in zip(lat, lat_at) if a >= warm]
    out["after_first_s"] = {"p99_ms": _latency_stats(steady)["p99_ms"] if steady else None,
                            "dropped_queue_full": sum(1 for x in drop_t if x >= 1.0)}
    out["submit_lag_ms_p99"] = float(np.percentile(np.asarray(lag, np.float64), 99)) * 1e-6 if lag else 0.0
    if len(rounds):
        busy = (rounds["done_ns"] - rounds["start_ns"]).astype(np.float64) * 1e-6
        setup = (rounds["setup_ns"] - rounds["start_ns"]).astype(np.float64) * 1e-6
        changed = (rounds["created"] > 0) | (rounds["retired"] > 0) | (rounds["replanned"] > 0)
        out["round_ms"] = {"p50": float(np.percentile(busy, 50)), "p99": float(np.percentile(busy, 99)),
                           "max": float(busy.max()), "of_last": int(len(rounds)),
                           "setup_rounds": int(changed.sum()),
                           "setup_max": float(setup.max()),
                           "setup_p99_of_setup_rounds": float(np.percentile(setup[changed], 99)) if changed.any() else 0.0}
    return out


def run_plain(trace: Trace, bank: FrameBank, n_learn: int = N_LEARN, max_backlog_s: float = 1.0) -> dict:
    """One synchronous hmi_process_frame per frame, in arrival order, from one
    thread; streams are created and learned before the trace starts.  A replay
    that falls more than max_backlog_s behind the trace stops there
    ("saturated"): its latency only grows from then on."""
    with _no_gc_pauses():
        return _run_plain(trace, bank, n_learn, max_backlog_s)


def _run_plain(trace: Trace, bank: FrameBank, n_learn: int, max_backlog_s: float) -> dict:
    lib = hmi.load()
    streams = {}
    for sp in trace.streams:
        s = hmi.Stream(sp.w, sp.h)
        s.learn(bank.learn_block(sp.src, n_learn))
        streams[sp.idx] = s
    handle = {k: s.handle for k, s in streams.items()}
    src = {sp.idx: sp.src for sp in trace.streams}
    at, ai, an = _arrivals(trace)
    lat = []
    ptr = hmi.hmi_pointer()
    pref = ctypes.byref(ptr)
    now = lib.hmi_server_now_ns
    proc = lib.hmi_process_frame
    errors, saturated = 0, False
    limit = int(max_backlog_s * 1e9)
    t0 = now()
    for t, idx, n in zip(at, ai, an):
        if n < n_learn:
            continue                          # learned up front
        due = t0 + int(t * 1e9)
        delay = due - now()
        if delay > 150_000:
            time.sleep((delay - 100_000) * 1e-9)
        elif -delay > limit:
            saturated = True
            break
        if proc(handle[idx], bank.frame_addr(src[idx], n, n_learn), None, pref) != hmi.HMI_OK:
            errors += 1
        lat.append((now() - due) * 1e-6)
    wall = (now() - t0) * 1e-9
    for s in streams.values():
        s.close()
    out = {"frames": len(lat), "frames_per_s": len(lat) / wall, "wall_s": wall, "errors": errors,
           "offered_frames_per_s": trace.frames / trace.duration, "saturated": saturated}
    out.update(_latency_stats(lat))
    return out


def run_plain_async(trace: Trace, bank: FrameBank, n_learn: int = N_LEARN, n_cuda_streams: int = 8,
                    max_backlog_s: float = 1.0) -> dict:
    """Asynchronous per-stream launches: streams learned up front; at its
    arrival time a frame is enqueued on CUDA stream idx mod n_cuda_streams as
    a host-to-device copy into its stream's device frame, an asynchronous
    per-frame call and a device-to-host copy of its pointer, closed by an
    event; a completion thread observes the events in submission order."""
    with _no_gc_pauses():
        return _run_plain_async(trace, bank, n_learn, n_cuda_streams, max_backlog_s)


def _run_plain_async(trace: Trace, bank: FrameBank, n_learn: int, n_cuda_streams: int,
                     max_backlog_s: float) -> dict:
    import collections
    import torch
    lib = hmi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    streams, dframe, dptr, hptr = {}, {}, {}, {}
    for sp in trace.streams:
        s = hmi.Stream(sp.w, sp.h)
        s.learn(bank.learn_block(sp.src, n_learn))
        streams[sp.idx] = s
        dframe[sp.idx] = torch.empty((sp.h, sp.w, 3), dtype=torch.uint8, device=dev)
        dptr[sp.idx] = torch.zeros(40, dtype=torch.uint8, device=dev)
        hptr[sp.idx] = torch.zeros(40, dtype=torch.uint8).pin_memory()
    css = [torch.cuda.Stream(device=dev) for _ in range(n_cuda_streams)]
    src = {sp.idx: sp.src for sp in trace.streams}
    at, ai, an = _arrivals(trace)
    now = lib.hmi_server_now_ns
    proc = lib.hmi_process_frame_async
    pending = collections.deque()
    cv = threading.Condition()
    lat, errors = [], [0]
    done_flag = [False]

    def completer():
        while True:
            with cv:
                while not pending and not done_flag[0]:
                    cv.wait(0.01)
                if not pending and done_flag[0]:
                    return
                ev, due = pending.popleft()
            ev.synchronize()
            lat.append((now() - due) * 1e-6)

    th = threading.Thread(target=completer, daemon=True)
    th.start()
    saturated = False
    limit = int(max_backlog_s * 1e9)
    t0 = now()
    for t, idx, n in zip(at, ai, an):
        if n < n_learn:
            continue                          # learned up front
        due = t0 + int(t * 1e9)
        delay = due - now()
        if delay > 150_000:
            time.sleep((delay - 100_000) * 1e-9)
        elif -delay > limit:
            saturated = True
            break
        cs = css[idx % n_cuda_streams]
        with torch.cuda.stream(cs):
            k = n - n_learn
            frame = bank.run[src[idx]][k % len(bank.run[src[idx]])]
            dframe[idx].copy_(frame.view(dframe[idx].shape), non_blocking=True)
            if proc(streams[idx].handle, dframe[idx].data_ptr(), None, dptr[idx].data_ptr(),
                    cs.cuda_stream) != hmi.HMI_OK:
                errors[0] += 1
            hptr[idx].copy_(dptr[idx], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cs)
        with cv:
            pending.append((ev, due))
            cv.notify()
    with cv:
        done_flag[0] = True
        cv.notify()
    th.join()
    wall = (now() - t0) * 1e-9
    torch.cuda.synchronize()
    for s in streams.values():
        s.close()
    out = {"frames": len(lat), "frames_per_s": len(lat) / wall, "wall_s": wall, "errors": errors[0],
           "offered_frames_per_s": trace.frames / trace.duration, "saturated": saturated,
           "cuda_streams": n_cuda_streams}
    out.update(_latency_stats(lat))
    return out


DROP_BUDGET = 0.01


def meets_slo(r: dict) -> bool:
    """p99 within SLO_MS, no errors, and at most DROP_BUDGET of the offered
    frames refused because a stream's queue was full."""
    offered = r["offered_frames_per_s"] * r["wall_s"]
    return (not r.get("saturated", False) and r["p99_ms"] <= SLO_MS and r.get("errors", 0) == 0 and
            r.get("dropped_queue_full", 0) <= DROP_BUDGET * offered)


def sweep(bank: FrameBank, rates, duration: float, n_learn: int = N_LEARN, seed: int = 1907043935,
          budget_bytes: int = 1 << 50):
    """Served and plain forms over the same traces at each arrival-rate scale
    (a device budget no trace reaches, so that only the serving form
    differs)."""
    # every rate's served run first, then the plain forms (they saturate from
    # the second rate on and leave host and device busy for a while after)
    traces = {r: make_trace(duration, rate_scale=r, seed=seed + int(r * 1000)) for r in rates}
    served = {r: run_served(traces[r], bank, budget_bytes, n_learn) for r in rates}
    rows = []
    for r in rates:
        pln = run_plain(traces[r], bank, n_learn)
        pla = run_plain_async(traces[r], bank, n_learn)
        rows.append({"rate_scale": r, "served": served[r], "plain": pln, "plain_async": pla})
    best = {}
    for arm in ("served", "plain", "plain_async"):
        ok = [row[arm]["frames_per_s"] for row in rows if meets_slo(row[arm])]
        best[arm] = max(ok) if ok else 0.0
    return rows, best
