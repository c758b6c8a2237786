"""The persistent tick's work queue (the planner in csrc/hmi_queue.h), on the CPU.

The kernel's CTAs take items in queue order, and an item waits only for its
stream's items of the step before (luma -> classify -> morphology strips).  The
launch ends for any grid size only if every stream's steps come in that order
in the queue; these tests build the planner with g++ and check that order,
that the items cover every chunk and strip exactly once, that the counts the
kernel waits for match, that the lag keeps a stream's classify items away from
its luma items, and, by simulating CTAs that take items in order (one fetched
ahead), that every item finishes.
"""
import os
import shutil
import subprocess

import pytest

from paper_1907_04393_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1907_04393_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"
MIX64 = [synth.shape(4, i) for i in range(synth.num_streams(4))]


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "vector_types.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("q") / "tick_queue_main")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-I", CUDA_INC,
                    os.path.join(ROOT, "tests", "native", "tick_queue_main.cpp"), "-o", exe],
                   check=True, capture_output=True)

    def run(shapes, piece=512, lag=0):
        args = [exe, str(piece), str(lag)]
        for w, h in shapes:
            args += [str(w), str(h)]
        out = subprocess.run(args, check=True, capture_output=True, text=True).stdout.split("\n")
        global STRIP_ROWS
        STRIP_ROWS = int(out[0].split()[1])
        items = [tuple(map(int, l.split())) for l in out[1:] if l and not l.startswith("sync")]
        sync = [tuple(map(int, l.split()[1:])) for l in out if l.startswith("sync")]
        return items, sync
    return run


STRIP_ROWS = 8


def geometry(w, h):
    nwords = (w + 31) // 32
    return h * 2 * nwords, -(-h // STRIP_ROWS) * ((nwords + 29) // 30)


def check_queue(shapes, items, sync, piece):
    pos = {}
    for i, (kind, s, b, e) in enumerate(items):
        pos.setdefault((s, kind), []).append((i, b, e))
    for s, (w, h) in enumerate(shapes):
        chunks, strips = geometry(w, h)
        for kind, n in ((0, chunks), (1, chunks), (2, strips)):
            rng = sorted((b, e) for _, b, e in pos[(s, kind)])
            assert rng[0][0] == 0 and rng[-1][1] == n
            assert all(a[1] == c[0] for a, c in zip(rng, rng[1:])), (s, kind)   # exact cover
        assert sync[s] == (len(pos[(s, 0)]), len(pos[(s, 1)]), len(pos[(s, 2)]))
        assert sync[s][0] == -(-chunks // piece)
        assert {k for (t, k) in pos if t == s} == {0, 1, 2}
        # every step after every item of the step before
        for k in range(2):
            assert max(i for i, _, _ in pos[(s, k)]) < min(i for i, _, _ in pos[(s, k + 1)]), (s, k)


def simulate(items, sync, ctas, dur):
    """CTAs take items in order (each holding its current item and one
    fetched ahead); an item runs when its stream has reached its step, for
    dur[kind] time units.  Returns the time at which the last item ends."""
    nstream = len(sync)
    stage = [0] * nstream
    done = [[0, 0, 0] for _ in range(nstream)]
    head, t = 0, 0
    slots = []                               # per CTA: [current, ahead, remaining time]
    for _ in range(ctas):
        cur = head if head < len(items) else None
        head += 1
        nxt = head if head < len(items) else None
        head += 1
        slots.append([cur, nxt, None])
    finished = 0
    while finished < len(items):
        t += 1
        assert t < 10 ** 7, "queue does not drain"
        progressed = False
        for sl in slots:
            if sl[0] is None:
                continue
            kind, s, _, _ = items[sl[0]]
            if sl[2] is None:
                if stage[s] < kind:
                    continue                 # waiting for the step before
                sl[2] = dur[kind]
            sl[2] -= 1
            progressed = True
            if sl[2] == 0:
                finished += 1
                done[s][kind] += 1
                if done[s][kind] == sync[s][kind]:
                    stage[s] = kind + 1
                sl[0], sl[2] = sl[1], None
                sl[1] = head if head < len(items) else None
                head += 1
        assert progressed or finished == len(items), "every CTA waits: deadlock"
    return t


def test_queue_order_and_cover_64_stream_mix(planner):
    for piece, lag in ((512, 0), (512, 912), (128, 300), (2048, 5)):
        items, sync = planner(MIX64, piece, lag)
        check_queue(MIX64, items, sync, piece)


def test_queue_lag_separates_luma_and_classify(planner):
    lag = 912
    items, sync = planner(MIX64, 512, lag)
    last_luma = max(i for i, it in enumerate(items) if it[0] == 0)
    lastL = {}
    for i, (kind, s, _, _) in enumerate(items):
        if kind == 0:
            lastL[s] = i
        elif kind == 1 and i < last_luma:     # before the tail every classify item keeps the lag
            assert i - lastL[s] >= lag
    # the frames held in L2 between a stream's luma and classify items stay
    # a small part of the 126 MB L2 (3 bytes per pixel, 16 px per chunk)
    open_chunks, peak = {}, 0
    for kind, s, b, e in items:
        if kind == 0:
            open_chunks[s] = open_chunks.get(s, 0) + (e - b)
        elif kind == 1:
            open_chunks[s] -= (e - b)
        peak = max(peak, sum(open_chunks.values()))
    assert peak * 16 * 3 < 40e6


def test_queue_drains_for_any_grid(planner):
    shapes = [(320, 240), (64, 64), (1920, 1080), (100, 37), (640, 480), (33, 1)]
    for lag in (0, 3, 50):
        items, sync = planner(shapes, 256, lag)
        check_queue(shapes, items, sync, 256)
        for ctas in (1, 2, 7, 64, 1000):
            simulate(items, sync, ctas, dur={0: 3, 1: 5, 2: 2})


def test_queue_single_stream(planner):
    items, sync = planner([(640, 480)], 512, 0)
    check_queue([(640, 480)], items, sync, 512)
    kinds = [it[0] for it in items]
    assert kinds == sorted(kinds)              # one stream: the steps in turn
    simulate(items, sync, 456, dur={0: 3, 1: 5, 2: 2})
