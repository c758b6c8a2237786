"""Run by tests/test_gpu_debug_build.py in a child process with
HMI_DEBUG_BUILD=1: the bounds-checked build of the library on tiny and ragged
frames through the per-frame path and the three forms of a batch tick, against the
CPU oracle, with guard bands around every output buffer (host and device)
that must come back untouched.  A failed bounds check in a kernel surfaces as
HMI_ERR_DEVICE (an exception here).  Prints "ok"."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1907_04393_gb300 import build, hmi  # noqa: E402

GUARD = 64          # bytes of guard band on each side (a multiple of 16)
FILL = 0xA5


def guarded_host(nbytes):
    buf = np.full(nbytes + 2 * GUARD, FILL, np.uint8)
    return buf, buf[GUARD:GUARD + nbytes]


def guarded_dev(nbytes):
    buf = torch.full((nbytes + 2 * GUARD,), FILL, dtype=torch.uint8, device="cuda")
    return buf, buf[GUARD:GUARD + nbytes]


def guards_intact(buf):
    a = buf.cpu().numpy() if hasattr(buf, "cpu") else buf
    return bool((a[:GUARD] == FILL).all() and (a[-GUARD:] == FILL).all())


def main():
    lib = hmi.load()
    assert lib._name == build.LIB_DEBUG, lib._name
    rng = np.random.default_rng(5)
    shapes = [(1, 1), (17, 5), (33, 33), (100, 75), (321, 241), (64, 48), (32, 64)]
    pairs = []
    for w, h in shapes:
        lf = rng.integers(0, 256, size=(3, h, w, 3), dtype=np.uint8)
        g, o = hmi.Stream(w, h), oracle.OracleStream(w, h)
        g.learn(lf)
        o.learn(lf)
        pairs.append((g, o))
    # the per-frame path, host buffers with guard bands
    for g, o in pairs:
        for _ in range(2):
            frame = rng.integers(0, 256, size=(g.h, g.w, 3), dtype=np.uint8)
            mbuf, mask = guarded_host(g.w * g.h)
            pbuf, pview = guarded_host(40)
            st = lib.hmi_process_frame(g.handle, frame.ctypes.data, mask.ctypes.data, pview.ctypes.data)
            assert st == hmi.HMI_OK, hmi.hmi_status_string(st)
            lbuf, lab = guarded_host(4 * g.w * g.h)
            hmi.hmi_get_labels(g.handle, lab.ctypes.data)
            m_o, l_o, p_o, _ = o.process(frame)
            assert np.array_equal(mask.reshape(g.h, g.w), m_o), (g.w, g.h)
            assert np.array_equal(lab.view(np.int32).reshape(g.h, g.w), l_o), (g.w, g.h)
            p = pview.view(hmi.POINTER_DTYPE)[0]
            assert int(p["area"]) == p_o["area"] and int(p["label"]) == p_o["label"]
            assert guards_intact(mbuf) and guards_intact(pbuf) and guards_intact(lbuf)
    # the three forms of a batch tick, device buffers with guard bands
    b = hmi.hmi_batch_create([g.handle for g, _ in pairs])
    try:
        for fused in (0, 1, 2):
            hmi.hmi_batch_set_tuning(b, dict(hmi.hmi_batch_get_tuning(b), fused=fused, groups=0,
                                             piece_chunks=32))
            frames = [rng.integers(0, 256, size=(g.h, g.w, 3), dtype=np.uint8) for g, _ in pairs]
            bufs = [guarded_dev(g.w * g.h) for g, _ in pairs]
            pbuf, pview = guarded_dev(40 * len(pairs))
            hmi.hmi_batch_process_async(b, [torch.from_numpy(f).cuda() for f in frames], [m for _, m in bufs],
                                        pview.data_ptr(), torch.cuda.current_stream().cuda_stream, True)
            torch.cuda.synchronize()
            ptrs = pview.cpu().numpy().view(hmi.POINTER_DTYPE)
            for i, (g, o) in enumerate(pairs):
                m_o, l_o, p_o, _ = o.process(frames[i])
                assert np.array_equal(bufs[i][1].cpu().numpy().reshape(g.h, g.w), m_o), (fused, g.w, g.h)
                assert np.array_equal(g.labels(), l_o), (fused, g.w, g.h)
                assert int(ptrs[i]["area"]) == p_o["area"] and int(ptrs[i]["label"]) == p_o["label"]
                assert guards_intact(bufs[i][0])
            assert guards_intact(pbuf)
            # a synchronous call returns any flag the ticks raised (none)
            hmi.hmi_batch_process(b, frames, None, None)
            for i, (g, o) in enumerate(pairs):
                o.process(frames[i])
    finally:
        hmi.hmi_batch_destroy(b)
        for g, _ in pairs:
            g.close()
    print("ok")


if __name__ == "__main__":
    main()
