"""Throughput benchmark of the hand-isolation path (arXiv 1907.04393) on GB300.

One step = one tick of the 64-stream batch: one frame for each of 64 camera
streams of mixed resolution (32 x 320x240, 16 x 640x480, 12 x 1280x720,
4 x 1920x1080; 26.7 Mpx), through every stage of the path (brightness gain,
background / gray / hue masks, morphology, components, pointer + click),
replayed from a CUDA graph on the current torch stream.  Inputs are resident
in HBM in a ring of 4 ticks per stream (320 MB, larger than the 126 MB L2).

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (on
the host cores, bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s & Mpixel/s at 640x480 and 64-stream batch; % HBM peak; p99 frame latency"
CFG = 4
RING = 4
# untimed ticks before the warm-up of each timed leg: a plan keeps a ring of 12
# per-tick slots, each with its own CUDA graph built on its first use, so two
# turns of the ring build and upload every graph before anything is timed
GRAPH_PRIME_TICKS = 24
WORKLOAD = ("64-stream batch: 32x320x240 + 16x640x480 + 12x1280x720 + 4x1920x1080 RGB8, "
            "26.7 Mpx per tick, each stream with its own learned background")
# algorithmic bytes per pixel of the classification (background, gray and hue
# test) kernel: frame 3 B + band lo/hi 6 B read, 1 bit written
CLASSIFY_BYTES_PER_PX = 3 + 6 + 1 / 8
# algorithmic bytes per pixel of the whole per-pixel stage (luma, band, gray /
# hue, morphology): the frame read once (3 B), the band (6 B), the 0/1 mask (1 B)
K2_BYTES_PER_PX = 3 + 6 + 1
# per-pixel kernels of a tick in the chained form (kernel indices of a tick):
# the band streams' gray and hue tests run inside the classify kernel, so the
# skin kernel launches only for mixture streams
K2_KERNELS = ("luma", "classify", "morphology")
# the one launch of the per-pixel stage in the other tick forms (hmi_tuning.fused)
FUSED_KERNEL = {1: "k_tick", 2: "k_stage"}
KERNELS_PER_TICK = 5          # per stream group: luma, classify, morphology, blocks, finish
# the Gaussian mixture background with its default 3 components: frame 3 B,
# 12 B of state per component read and written, 1 bit written
MIX_BENCH = dict(bg_model=1, mix_k=3)
MIX_BYTES_PER_PX = 3 + 2 * 12 * MIX_BENCH["mix_k"] + 1 / 8
# per background model: the per-pixel kernel, its algorithmic bytes per pixel,
# its committed ncu summary and the sources its hash covers
BG_MODELS = {
    "band": dict(params={}, kernel="classify", bytes_per_px=CLASSIFY_BYTES_PER_PX,
                 profile=os.path.join(ROOT, "profiles", "k_classify_64stream.txt"),
                 sources=("hmi_frame.cu", "hmi_pixel.cuh", "hmi_band.h", "hmi_internal.cuh", "hmi_queue.h")),
    "mixture": dict(params=MIX_BENCH, kernel="mixture", bytes_per_px=MIX_BYTES_PER_PX,
                    profile=os.path.join(ROOT, "profiles", "k_mix_64stream.txt"),
                    sources=("hmi_mix.cu", "hmi_internal.cuh")),
}


# --------------------------------------------------------------------------- #
# helpers                                                                      #
# --------------------------------------------------------------------------- #
def peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(sources=BG_MODELS["band"]["sources"]) -> str:
    """Hash of a per-pixel kernel's code (comments and blank lines left out,
    so that a comment edit does not orphan the committed counters)."""
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_1907_04393_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic_per_px(model: str = "band"):
    """DRAM bytes per pixel of the model's per-pixel kernel from the committed
    ncu summary, if it was taken on the current kernel source."""
    m = BG_MODELS[model]
    try:
        kv = {}
        with open(m["profile"]) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_hash") != kernel_source_hash(m["sources"]):
            return None
        return float(kv["dram_bytes_per_px"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        rows = [r for (t, r) in self.rows if t0 - 0.15 <= t <= t1 + 0.15] or [r for _, r in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if len(r) > 8 and num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if len(r) > 8 and num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) > 8 for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        pw = [num(r[3]) for r in rows if len(r) > 8 and num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


# --------------------------------------------------------------------------- #
# CPU oracle workers (spawned processes, no CUDA in them)                      #
# --------------------------------------------------------------------------- #
def _oracle_serve(conn, cfg, owned):
    """Owns `owned` streams: learns them once, then on ("run", t, count)
    processes `count` stream-frames round robin over its streams (frames of
    tick t, generated before the clock starts) and returns (frames, px, s)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle
    from paper_1907_04393_gb300 import synth
    streams = []
    for s in owned:
        o = oracle.OracleStream(*synth.shape(cfg, s))
        o.learn(synth.learn_frames(cfg, s))
        streams.append((s, o))
    conn.send("ready")
    nxt = 0
    while True:
        msg = conn.recv()
        if msg[0] == "stop":
            break
        _, t, count = msg
        work = []
        for _ in range(count):
            s, o = streams[nxt % len(streams)]
            nxt += 1
            work.append((o, synth.run_frame(cfg, s, t)))
        start = time.perf_counter()
        px = 0
        for o, fr in work:
            o.process(fr, want_labels=False)
            px += o.w * o.h
        conn.send((len(work), px, time.perf_counter() - start))


class OraclePool:
    """The oracle as it stands (single threaded), one spawned process per core,
    each owning a fixed share of the workload's streams."""

    def __init__(self, cfg: int, n_streams: int, workers: int, owned=None):
        ctx = mp.get_context("spawn")
        self.owned = owned if owned is not None else [list(range(j, n_streams, workers)) for j in range(workers)]
        self.owned = [o for o in self.owned if o]
        self.conns, self.procs = [], []
        for o in self.owned:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_serve, args=(b, cfg, o), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"

    @property
    def cores(self) -> int:
        return len(self.procs)

    def run(self, t: int, per_worker: int | None = None) -> dict:
        """One round: every worker processes per_worker stream-frames (None: all
        of its streams, i.e. one full tick).  Time = the slowest worker."""
        for c, o in zip(self.conns, self.owned):
            c.send(("run", t, len(o) if per_worker is None else per_worker))
        res = [c.recv() for c in self.conns]
        return {"frames": sum(r[0] for r in res), "px": sum(r[1] for r in res),
                "seconds": max(r[2] for r in res)}

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)


def copy_same_bytes_us(nbytes: int, reps: int = 10) -> float:
    """Median time of a plain device-to-device copy that moves nbytes in all
    (nbytes / 2 read, nbytes / 2 written), L2 flushed before each: what HBM
    gives one kernel of that traffic on this GPU, launch ramp and tail
    included.  The measured peak comes from a multi-GiB copy; kernels of a
    few hundred MB reach a smaller share of it."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    half = max(nbytes // 2, 1 << 20)
    src = torch.empty(half, dtype=torch.uint8, device=dev).fill_(1)
    dst = torch.empty_like(src)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ts = []
    for _ in range(reps):
        flush.fill_(0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dst.copy_(src)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e3)
    del src, dst, flush
    ts.sort()
    return ts[len(ts) // 2]


def k2_roofline(per_kernel: dict, ticks: int, px: int, fused: bool, peak: float, peak_kind: str) -> dict:
    """The per-pixel stage against HBM: K2_BYTES_PER_PX x px over the summed
    CUDA-event times of its kernels (the persistent tick's one launch when
    fused), from a single-chain pass where each kernel is timed alone.  Beside
    it, a plain copy of the same traffic timed the same way (one launch)."""
    names = ("luma",) if fused else K2_KERNELS
    ms = sum(per_kernel[k] for k in names) / max(ticks, 1)
    nbytes = K2_BYTES_PER_PX * px
    achieved = nbytes / (ms / 1e3) / 1e9
    copy_us = copy_same_bytes_us(nbytes)
    # the same for each kernel's own traffic: frame (3 B/px); frame, band and
    # raw bits (9.125 B/px); raw bits in, bits and mask bytes out (1.25 B/px)
    per_copy = {} if fused else {k: copy_same_bytes_us(int(bpp * px))
                                 for k, bpp in (("luma", 3.0), ("classify", 9.125), ("morphology", 1.25))}
    return {"bound": "hbm", "kernels": [FUSED_KERNEL[int(fused)]] if fused else ["k_luma", "k_classify", "k_morph_strip"],
            "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": achieved / peak, "algorithmic_bytes_per_tick": nbytes,
            "bytes_per_px": K2_BYTES_PER_PX, "stage_ms": ms, "ticks_timed": ticks,
            "copy_same_bytes": {"us": copy_us, "GBs": nbytes / copy_us / 1e3,
                                "frac_of_peak": nbytes / copy_us / 1e3 / peak,
                                "stage_over_copy": ms * 1e3 / copy_us},
            "copy_per_kernel_traffic_us": per_copy,
            "stage_over_per_kernel_copies": (ms * 1e3 / sum(per_copy.values())) if per_copy else None}


def max_over_ranks(x: float, dev) -> float:
    """The slowest rank's time (every rank gets it); x itself with one rank."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest
    rank's time (weak scaling: each rank runs the same workload)."""
    return units_per_rank * world / (ms / 1e3)


def host_workers(n_streams: int) -> int:
    return max(1, min(os.cpu_count() or 1, 16, n_streams))


# --------------------------------------------------------------------------- #
# reference arm: the CPU oracle on the host cores                              #
# --------------------------------------------------------------------------- #
def run_reference(args) -> None:
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from paper_1907_04393_gb300 import synth
    n = synth.num_streams(CFG)
    pool = OraclePool(CFG, n, host_workers(n))
    try:
        # one step = one stream-frame per core (round robin over the 64 streams)
        for k in range(max(args.warmup, 1)):
            pool.run(k, 1)
        budget, t_start = 150.0, time.time()
        done, frames, px, secs = 0, 0, 0, 0.0
        while done < args.steps and (time.time() - t_start) < budget:
            r = pool.run(args.warmup + done, 1)
            frames, px, secs, done = frames + r["frames"], px + r["px"], secs + r["seconds"], done + 1
    finally:
        pool.close()
    fps = frames / secs
    sample = f"{pool.cores} stream-frames per step (one per core, round robin over the 64 streams)"
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": done, "warmup": args.warmup,
        "ms_per_step": secs / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "mpx_per_s": px / secs / 1e6,
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": pool.cores, "kind": "oracle",
                         "sample": f"{sample}; {done} steps"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# our arm                                                                      #
# --------------------------------------------------------------------------- #
def run_ours(args) -> None:
    import torch
    import torch.distributed as dist
    from paper_1907_04393_gb300 import hmi, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    hmi.load()
    # ---- serving: 256-stream arrival trace (rank 0 of a 1-GPU run), first of
    # all, in a fresh process: its latency tails come from host threads ------
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        serving = bench_serving(hmi, args)
        torch.cuda.empty_cache()

    # CPU baseline after the serving workload (spawned processes: no CUDA
    # state of this process reaches them)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(CFG, synth.num_streams(CFG), host_workers(synth.num_streams(CFG)))
        try:
            pool.run(0)                                   # warm-up tick
            rs = [pool.run(1 + k) for k in range(args.cpu_ticks)]
        finally:
            pool.close()
        cpu = {"frames": sum(r["frames"] for r in rs), "px": sum(r["px"] for r in rs),
               "seconds": sum(r["seconds"] for r in rs), "cores": pool.cores}
        # the oracle on one core: one process owning a sample of the mix (four
        # 320x240, two 640x480, one 1280x720 and one 1920x1080 stream), each
        # stream-frame timed once
        one = OraclePool(CFG, synth.num_streams(CFG), 1, owned=[list(SINGLE_CORE_SAMPLE)])
        try:
            one.run(0)
            r1 = [one.run(1 + k) for k in range(2)]
        finally:
            one.close()
        cpu["single"] = {"frames": sum(r["frames"] for r in r1), "px": sum(r["px"] for r in r1),
                         "seconds": sum(r["seconds"] for r in r1)}


    n = synth.num_streams(CFG)
    streams, rings, masks = [], [], []
    px_per_tick = 0
    for i in range(n):
        w, h = synth.shape(CFG, i)
        st = hmi.Stream(w, h, **BG_MODELS[args.bg_model]["params"])
        st.learn(torch.from_numpy(synth.learn_frames(CFG, i)).to(dev))
        streams.append(st)
        rings.append([torch.from_numpy(synth.run_frame(CFG, i, t)).to(dev) for t in range(RING)])
        masks.append(torch.empty((h, w), dtype=torch.uint8, device=dev))
        px_per_tick += w * h
    ptrs = torch.zeros(n * 40, dtype=torch.uint8, device=dev)
    batch = hmi.hmi_batch_create([s.handle for s in streams])
    default_groups = hmi.hmi_batch_get_groups(batch)
    pipelined = args.mode == "pipelined"
    if pipelined:
        hmi.hmi_batch_set_groups(batch, 1)      # pipelined ticks run as one chain
    elif args.groups:
        hmi.hmi_batch_set_groups(batch, args.groups)
    cs = torch.cuda.current_stream()

    # the frame and mask address arrays of each ring position, built once
    ring_arrs = [hmi.ptr_array(rings[i][r] for i in range(n)) for r in range(RING)]
    mask_arr = hmi.ptr_array(masks)

    def tick(k):
        hmi.hmi_batch_process_async(batch, ring_arrs[k % RING], mask_arr, ptrs.data_ptr(), cs.cuda_stream, True)

    def tick_main(k):
        if pipelined:
            hmi.hmi_batch_process_pipelined(batch, ring_arrs[k % RING], mask_arr,
                                            ptrs.data_ptr(), cs.cuda_stream, True)
        else:
            tick(k)

    def finish_main():
        if pipelined:
            hmi.hmi_batch_flush(batch, cs.cuda_stream)   # the last tick's second stage

    if args.fused >= 0:
        hmi.hmi_batch_set_tuning(batch, dict(hmi.hmi_batch_get_tuning(batch), fused=args.fused))
    # launch shape: searched by the library's autotuner (untimed), or the default
    tuned = None
    if not args.no_autotune:
        from paper_1907_04393_gb300 import autotune
        shapes = [synth.shape(CFG, i) for i in range(n)]
        tuned = autotune.tune(batch, shapes, [rings[i][0] for i in range(n)],
                              torch.cuda.get_device_name(dev), pipelined, ticks=50, cache_path=None)
    shape_used = hmi.hmi_batch_get_tuning(batch)

    for k in range(GRAPH_PRIME_TICKS):
        tick_main(k)
    finish_main()
    for k in range(args.warmup):
        tick_main(k)
    finish_main()
    torch.cuda.synchronize()

    gpu_id = str(local)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    time.sleep(0.3)

    # ---- device-resident timed region ------------------------------------
    groups = hmi.hmi_batch_get_groups(batch)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(cs)
    for k in range(args.steps):
        tick_main(args.warmup + k)
    finish_main()
    e1.record(cs)
    torch.cuda.synchronize()
    barrier()
    t1 = time.time()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    clk = clocks.summary(t0, t1)
    clocks.stop()

    # ---- plain (unpipelined) ticks with the library's default groups ------
    plain_steps = max(10, min(args.steps, 2000))
    hmi.hmi_batch_set_groups(batch, args.groups or default_groups)
    plain_groups = hmi.hmi_batch_get_groups(batch)
    for k in range(GRAPH_PRIME_TICKS + args.warmup):
        tick(k)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(cs)
    for k in range(plain_steps):
        tick(args.warmup + k)
    q1.record(cs)
    torch.cuda.synchronize()
    plain_ms = q0.elapsed_time(q1) / plain_steps

    # ---- roofline pass: the same ticks with one chain, so that each
    # classification launch is timed alone with events on its stream -------
    hmi.hmi_batch_set_groups(batch, 1)
    for k in range(GRAPH_PRIME_TICKS + args.warmup):
        tick(k)
    torch.cuda.synchronize()
    roof_steps = max(10, min(args.steps, 1000))
    hmi.hmi_batch_profile(batch, roof_steps)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(cs)
    for k in range(roof_steps):
        tick(args.warmup + k)
    r1.record(cs)
    torch.cuda.synchronize()
    one_chain_ms = r0.elapsed_time(r1) / roof_steps
    prof_ticks, per_kernel = hmi.hmi_batch_profile_kernels(batch)
    model = BG_MODELS[args.bg_model]
    fused_main = int(hmi.hmi_batch_get_tuning(batch)["fused"])   # 0: the chain
    prof_ms = per_kernel["luma" if fused_main else model["kernel"]]
    hmi.hmi_batch_profile(batch, 0)

    # ---- the other forms of the tick (chain, persistent launch, cooperative
    # stage), timed the same way, for the record ------------------------------
    other = None
    if args.bg_model == "band" and world == 1 and not args.no_other_form:
        other = [bench_other_form(hmi, batch, rings, masks, ptrs, cs, n, px_per_tick, args, f)
                 for f in (0, 1, 2) if f != fused_main]
    hmi.hmi_batch_set_tuning(batch, dict(shape_used, groups=plain_groups))

    # ---- end to end through the synchronous API with host buffers --------
    host_frames = []
    for i in range(n):
        host_frames.append([r.cpu().pin_memory() for r in rings[i]])
    host_ptrs = np.zeros(n, hmi.POINTER_DTYPE)
    host_arrs = [hmi.ptr_array(host_frames[i][r] for i in range(n)) for r in range(RING)]
    e2e_steps = max(3, min(args.steps, args.e2e_steps))
    for k in range(3):
        hmi.hmi_batch_process(batch, host_arrs[k % RING], mask_arr, host_ptrs)
    barrier()
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    for k in range(e2e_steps):
        hmi.hmi_batch_process(batch, host_arrs[k % RING], mask_arr, host_ptrs)
    e2e_sync_s = max_over_ranks(time.perf_counter() - s0, dev)
    # the same with every mask copied back to pinned host memory too
    host_masks = [torch.empty((m.shape[0], m.shape[1]), dtype=torch.uint8).pin_memory().numpy() for m in masks]
    host_mask_arr = hmi.ptr_array(host_masks)
    for k in range(3):
        hmi.hmi_batch_process(batch, host_arrs[k % RING], host_mask_arr, host_ptrs)
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    for k in range(e2e_steps):
        hmi.hmi_batch_process(batch, host_arrs[k % RING], host_mask_arr, host_ptrs)
    e2e_mask_s = max_over_ranks(time.perf_counter() - s0, dev)
    mask_bytes = sum(int(m.size) for m in host_masks)
    h2d = sum(int(host_frames[i][0].numel()) for i in range(n))

    # ---- end to end through the pipelined API: the same pinned host frames
    # (read by the luma pass over the host link), every step's pointers
    # copied back to pinned host memory --------------------------------------
    hmi.hmi_batch_set_groups(batch, 1)
    dptrs = torch.zeros(n * 40, dtype=torch.uint8, device=dev)
    hptrs = torch.zeros(n * 40, dtype=torch.uint8).pin_memory()

    def e2e_step(k):
        hmi.hmi_batch_process_pipelined(batch, host_arrs[k % RING], mask_arr,
                                        dptrs.data_ptr(), cs.cuda_stream, True)
        hptrs.copy_(dptrs, non_blocking=True)

    # the launch shape for host frames (the luma pass now also moves the frames
    # over the host link): the library's autotuner on these frames, untimed
    e2e_shape, _ = hmi.hmi_batch_autotune(batch, [host_frames[i][0] for i in range(n)], 30, True)
    e2e_depth = e2e_shape["pipeline_depth"]
    for k in range(GRAPH_PRIME_TICKS + max(3, args.warmup)):
        e2e_step(k)
    hmi.hmi_batch_flush(batch, cs.cuda_stream)
    torch.cuda.synchronize()
    barrier()
    s0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_step(k)
    hmi.hmi_batch_flush(batch, cs.cuda_stream)
    hptrs.copy_(dptrs, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - s0, dev)
    hmi.hmi_batch_set_tuning(batch, dict(shape_used, groups=plain_groups))

    # ---- re-learning on every stream: its cost on the same workload -------
    relearn = None
    # (the extra measurements below run on one-GPU runs only: a multi-GPU run
    # holds every GPU, and its line reports the scaled main workload)
    extras = world == 1
    if extras and not args.no_relearn:
        relearn = bench_relearn_cost(hmi, synth, torch, dev, cs, rings, shape_used, args)

    # ---- the Gaussian mixture background on every stream ------------------
    mixture = None
    if extras and not args.no_mixture and args.bg_model == "band":
        mixture = bench_mixture_cost(hmi, synth, torch, dev, cs, rings, shape_used, args)

    # ---- background quality under drift: band, re-learning, mixture -------
    quality = None
    if extras and args.quality_frames:
        quality = bench_background_quality(hmi, synth, torch, dev, args.quality_frames)

    # ---- single 640x480 stream (the other configuration of the metric) ---
    single = None
    if extras and not args.no_single:
        single = bench_single(hmi, synth, torch, dev, cs, args, 2)
        single_hd = bench_single(hmi, synth, torch, dev, cs, args, 3)

    hmi.hmi_batch_destroy(batch)
    for s in streams:
        s.close()
    for r in rings:
        r.clear()
    torch.cuda.empty_cache()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    value = whole_job_rate(n * args.steps, world, ms)
    classify_ms = prof_ms / max(prof_ticks, 1)
    roof_bytes_px = K2_BYTES_PER_PX if fused_main else model["bytes_per_px"]
    achieved = roof_bytes_px * px_per_tick / (classify_ms / 1e3) / 1e9
    traffic_px = None if fused_main else profiled_traffic_per_px(args.bg_model)
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "streams_per_gpu": n, "px_per_tick": px_per_tick,
                   "l2": f"inputs larger than L2: ring of {RING} ticks per stream "
                         f"({RING * px_per_tick * 3 / 1e6:.0f} MB of frames)",
                   "launch": ("pipelined ticks: one CUDA graph per tick on the torch current stream "
                              "runs stage 1 (gains, band test) of tick k beside stage 2 (gray/hue, "
                              "morphology, components, pointer) of tick k-1; one flush ends the timed "
                              "region" if pipelined else
                              f"CUDA graph per tick on the torch current stream, {groups} overlapping "
                              "stream groups"),
                   "graph_priming": f"{GRAPH_PRIME_TICKS} untimed ticks before the warm-up build and upload "
                                    "the CUDA graph of each of the plan's 12 per-tick slots"},
        "tuning": {"shape": shape_used,
                   "autotuned": tuned is not None,
                   "search_tick_us": None if tuned is None else tuned["tick_us"]},
        "plain_ticks": {"ms_per_step": plain_ms, "frames_per_s": n * world / (plain_ms / 1e3),
                        "groups": plain_groups, "steps": plain_steps,
                        "launch": "hmi_batch_process_async, one CUDA graph per tick"},
        "mpx_per_s": px_per_tick * args.steps * world / (ms / 1e3) / 1e6,
        "roofline": {"bound": "hbm",
                     "kernel": FUSED_KERNEL[fused_main] if fused_main else "k_" + ("classify" if args.bg_model == "band" else "mix<3>"),
                     "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": (traffic_px * px_per_tick) if traffic_px else None,
                     "algorithmic_bytes_per_launch": roof_bytes_px * px_per_tick,
                     "launch_ms": classify_ms, "launches_timed": prof_ticks,
                     "timed_in": "single-chain pass of the same workload, CUDA events around the "
                                 f"{FUSED_KERNEL[fused_main] if fused_main else model['kernel']} kernel alone "
                                 "(no other kernel overlaps it)",
                     "single_chain_ms_per_step": one_chain_ms,
                     "single_chain_kernels_us": {k: v / max(prof_ticks, 1) * 1e3 for k, v in per_kernel.items()}},
        "k2": k2_roofline(per_kernel, prof_ticks, px_per_tick, fused_main, peak, peak_kind)
              if args.bg_model == "band" else None,
        "e2e": {"value": n * e2e_steps * world / e2e_s, "unit": "frames/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": n * 40,
                "h2d_GBps": h2d * e2e_steps / e2e_s / 1e9, "pipeline_depth": e2e_depth,
                "tuning": e2e_shape,
                "api": "hmi_batch_process_pipelined on the torch current stream: pinned host frames "
                       "(read over the host link by the luma pass, no copy engine), every step's "
                       "pointers copied back to pinned host memory; wall clock, flush and a final "
                       "synchronize inside the timed region; launch shape autotuned on the host frames",
                "sync": {"value": n * e2e_steps * world / e2e_sync_s, "unit": "frames/s",
                         "api": "hmi_batch_process (synchronous), same host buffers, host pointers"},
                "sync_host_masks": {"value": n * e2e_steps * world / e2e_mask_s, "unit": "frames/s",
                                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": mask_bytes + n * 40,
                                    "api": "hmi_batch_process (synchronous), pinned host frames, every "
                                           "0/1 mask and pointer copied back to pinned host memory"}},
        "gpu_launches": (3 if fused_main else KERNELS_PER_TICK) * groups * args.steps,
        "clocks": clk,
    }
    if single is not None:
        line["single_640x480"] = single
        line["single_1920x1080"] = single_hd
    if other is not None:
        line["other_tick_forms"] = other
    if args.bg_model != "band":
        line["config"]["background"] = dict(MIX_BENCH)
    if relearn is not None:
        line["adaptive"] = relearn
    if mixture is not None:
        line["mixture"] = mixture
    if quality is not None:
        line["background_quality"] = quality
    if serving is not None:
        line["serving"] = serving
    if cpu is not None:
        line["cpu_baseline"] = {"value": cpu["frames"] / cpu["seconds"], "unit": "frames/s",
                                "cores": cpu["cores"], "kind": "oracle",
                                "sample": f"{cpu['frames']} stream-frames ({args.cpu_ticks} ticks of "
                                          f"all 64 streams), {cpu['px'] / 1e6:.0f} Mpx",
                                "mpx_per_s": cpu["px"] / cpu["seconds"] / 1e6,
                                "single_thread": {
                                    "frames_per_s": cpu["single"]["frames"] / cpu["single"]["seconds"],
                                    "mpx_per_s": cpu["single"]["px"] / cpu["single"]["seconds"] / 1e6,
                                    "cores": 1,
                                    "sample": f"{cpu['single']['frames']} stream-frames: 2 rounds over streams "
                                              f"{list(SINGLE_CORE_SAMPLE)} of the mix (4x320x240, 2x640x480, "
                                              f"1x1280x720, 1x1920x1080), "
                                              f"{cpu['single']['px'] / 1e6:.1f} Mpx"}}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


RELEARN_BENCH = dict(relearn_frames=30, relearn_min=20, relearn_period=300)
# streams of the 64-stream mix for the one-core oracle timing, in the mix's own
# proportions of sizes (indices 0-31: 320x240, 32-47: 640x480, 48-59:
# 1280x720, 60-63: 1920x1080)
SINGLE_CORE_SAMPLE = (0, 8, 16, 24, 32, 40, 48, 60)
TRACK_BENCH = 64


FORM_NAMES = {0: "chain of kernels",
              1: "persistent tick (one launch for luma, band/gray/hue and morphology items)",
              2: "cooperative per-pixel stage (one launch, luma / band, gray, hue / morphology "
                 "phases between grid barriers)"}


def bench_other_form(hmi, batch, rings, masks, ptrs, cs, n, px, args, form) -> dict:
    """The 64-stream batch with another form of the tick (hmi_tuning.fused:
    0 the chain, 1 the persistent launch, 2 the cooperative stage; the best
    piece size of a short search for the one-launch forms).  Pipelined ticks,
    then a single-chain pass with its per-pixel stage timed by CUDA events."""
    import torch
    peak, peak_kind = peaks()
    base = dict(hmi.hmi_batch_get_tuning(batch), groups=1, fused=form)
    fused_main = form == 0

    def pipelined(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(GRAPH_PRIME_TICKS + args.warmup):
            hmi.hmi_batch_process_pipelined(batch, [rings[i][k % RING] for i in range(n)], masks,
                                            ptrs.data_ptr(), cs.cuda_stream, True)
        hmi.hmi_batch_flush(batch, cs.cuda_stream)
        torch.cuda.synchronize()
        e0.record(cs)
        for k in range(steps):
            hmi.hmi_batch_process_pipelined(batch, [rings[i][k % RING] for i in range(n)], masks,
                                            ptrs.data_ptr(), cs.cuda_stream, True)
        hmi.hmi_batch_flush(batch, cs.cuda_stream)
        e1.record(cs)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    steps = max(20, min(args.steps, 500))
    best = None
    for piece in ((1024, 2048, 4096) if not fused_main else (base["piece_chunks"],)):
        t = dict(base, piece_chunks=piece)
        hmi.hmi_batch_set_tuning(batch, t)
        ms = pipelined(steps)
        if best is None or ms < best[1]:
            best = (t, ms)
    hmi.hmi_batch_set_tuning(batch, best[0])
    hmi.hmi_batch_profile(batch, steps)
    for k in range(steps):
        hmi.hmi_batch_process_async(batch, [rings[i][k % RING] for i in range(n)], masks, ptrs.data_ptr(),
                                    cs.cuda_stream, True)
    ticks, per = hmi.hmi_batch_profile_kernels(batch)
    hmi.hmi_batch_profile(batch, 0)
    fused = int(best[0]["fused"])
    return {"form": FORM_NAMES[fused],
            "tuning": best[0], "pipelined_ms_per_step": best[1], "frames_per_s": n / (best[1] / 1e3),
            "k2": k2_roofline(per, ticks, px, fused, peak, peak_kind),
            "single_chain_kernels_us": {k: round(v / max(ticks, 1) * 1e3, 2) for k, v in per.items()}}


def bench_relearn_cost(hmi, synth, torch, dev, cs, rings, shape, args) -> dict:
    """The 64-stream batch again with the adaptive features on every stream:
    re-learning (a window of 30 frames every 300), tracking, and an interface
    (four zones and a wheel): pipelined ticks over whole periods, with the
    same launch shape, then one period of plain ticks timed kernel by kernel."""
    n = len(rings)
    p = hmi.hmi_default_params(**RELEARN_BENCH)
    streams = []
    for i in range(n):
        w, h = synth.shape(CFG, i)
        st = hmi.Stream(w, h, track_max_dist=TRACK_BENCH, **RELEARN_BENCH)
        st.learn(torch.from_numpy(synth.learn_frames(CFG, i)).to(dev))
        st.set_interface(hmi.make_interface(
            [(0, 0, w // 2 - 1, h // 2 - 1, 1), (w // 2, 0, w - 1, h // 2 - 1, 2),
             (0, h // 2, w // 2 - 1, h - 1, 3), (w // 2, h // 2, w - 1, h - 1, 4)],
            (w // 2, h // 2, h // 8, h // 2, 64)))
        streams.append(st)
    b = hmi.hmi_batch_create([s.handle for s in streams])
    hmi.hmi_batch_set_tuning(b, dict(shape, groups=1))
    masks = [torch.empty((s.h, s.w), dtype=torch.uint8, device=dev) for s in streams]
    ptrs = torch.zeros(n * 40, dtype=torch.uint8, device=dev)
    steps = 4 * p.relearn_period
    for k in range(p.relearn_period):
        hmi.hmi_batch_process_pipelined(b, [rings[i][k % RING] for i in range(n)], masks, ptrs.data_ptr(),
                                        cs.cuda_stream, True)
    hmi.hmi_batch_flush(b, cs.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    for k in range(steps):
        hmi.hmi_batch_process_pipelined(b, [rings[i][k % RING] for i in range(n)], masks, ptrs.data_ptr(),
                                        cs.cuda_stream, True)
    hmi.hmi_batch_flush(b, cs.cuda_stream)
    e1.record(cs)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # one period of plain ticks with every kernel timed alone
    hmi.hmi_batch_profile(b, p.relearn_period)
    for k in range(p.relearn_period):
        hmi.hmi_batch_process_async(b, [rings[i][k % RING] for i in range(n)], masks, ptrs.data_ptr(),
                                    cs.cuda_stream, True)
    ticks, per = hmi.hmi_batch_profile_kernels(b)
    hmi.hmi_batch_profile(b, 0)
    hmi.hmi_batch_destroy(b)
    for s in streams:
        s.close()
    return {"params": dict(RELEARN_BENCH, track_max_dist=TRACK_BENCH, interface="4 zones + wheel"),
            "ms_per_step": ms, "frames_per_s": n / (ms / 1e3),
            "steps": steps, "launch": "pipelined ticks, the main run's launch shape, one group",
            "per_period_ms": {k: round(v, 3) for k, v in per.items()}, "period_ticks": ticks,
            "sums_ms_per_window_tick": per["relearn"] / p.relearn_frames,
            "band_reform_ms_per_window_end": per["relearn_band"]}


def bench_mixture_cost(hmi, synth, torch, dev, cs, rings, shape, args) -> dict:
    """The 64-stream batch with the Gaussian mixture background (3 components)
    on every stream: pipelined ticks with the main run's launch shape, then
    plain ticks timed kernel by kernel, the mixture kernel against HBM."""
    n = len(rings)
    streams, px = [], 0
    for i in range(n):
        w, h = synth.shape(CFG, i)
        st = hmi.Stream(w, h, **MIX_BENCH)
        st.learn(torch.from_numpy(synth.learn_frames(CFG, i)).to(dev))
        streams.append(st)
        px += w * h
    b = hmi.hmi_batch_create([s.handle for s in streams])
    hmi.hmi_batch_set_tuning(b, dict(shape, groups=1))
    masks = [torch.empty((s.h, s.w), dtype=torch.uint8, device=dev) for s in streams]
    ptrs = torch.zeros(n * 40, dtype=torch.uint8, device=dev)
    steps = max(50, min(args.steps, 1000))

    def run(k0, count, pipelined):
        for k in range(k0, k0 + count):
            fr = [rings[i][k % RING] for i in range(n)]
            if pipelined:
                hmi.hmi_batch_process_pipelined(b, fr, masks, ptrs.data_ptr(), cs.cuda_stream, True)
            else:
                hmi.hmi_batch_process_async(b, fr, masks, ptrs.data_ptr(), cs.cuda_stream, True)
        if pipelined:
            hmi.hmi_batch_flush(b, cs.cuda_stream)

    run(0, max(args.warmup, 3), True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    run(0, steps, True)
    e1.record(cs)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = max(10, min(steps, 300))
    hmi.hmi_batch_profile(b, prof)
    run(0, prof, False)
    ticks, per = hmi.hmi_batch_profile_kernels(b)
    hmi.hmi_batch_profile(b, 0)
    hmi.hmi_batch_destroy(b)
    for st in streams:
        st.close()
    mix_ms = per["mixture"] / max(ticks, 1)
    peak, peak_kind = peaks()
    achieved = MIX_BYTES_PER_PX * px / (mix_ms / 1e3) / 1e9
    traffic_px = profiled_traffic_per_px("mixture")
    return {"params": dict(MIX_BENCH), "ms_per_step": ms, "frames_per_s": n / (ms / 1e3),
            "mpx_per_s": px / (ms / 1e3) / 1e6, "steps": steps,
            "launch": "pipelined ticks, the main run's launch shape, one group",
            "roofline": {"bound": "hbm", "kernel": "k_mix<3>", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (traffic_px * px) if traffic_px else None,
                         "algorithmic_bytes_per_launch": MIX_BYTES_PER_PX * px,
                         "launch_ms": mix_ms, "launches_timed": ticks},
            "single_chain_kernels_us": {k: round(v / max(ticks, 1) * 1e3, 2) for k, v in per.items()}}


# the gray and hue tests opened to every coloured pixel and morphology off, so
# that the final mask is the background test's own decision
BG_TEST_ONLY = dict(gray_tol=0, hue_lo=0, hue_hi=1535, open_iters=0, close_iters=0)


def bench_background_quality(hmi, synth, torch, dev, frames: int) -> dict:
    """1920x1080 drifting scene (the third single-stream workload: gradient
    drift of one level per 50 frames, brightness flicker, two moving hands)
    with three background models: the learned band alone, the band with
    re-learning, and the Gaussian mixture; the gray/hue tests and morphology
    are neutral, so the mask is the background test's decision.  At every
    100th frame: the share of non-hand pixels the test calls foreground (false
    foreground) and the share of hand pixels it calls foreground (recall)."""
    import numpy as np
    w, h = synth.shape(3)
    lf = torch.from_numpy(synth.learn_frames(3, 0)).to(dev)
    models = {"band": {}, "band_relearn": RELEARN_BENCH, "mixture": MIX_BENCH}
    streams = {}
    for name, over in models.items():
        st = hmi.Stream(w, h, **BG_TEST_ONLY, **over)
        st.learn(lf)
        streams[name] = st
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float32)
    false_fg = {k: [] for k in models}
    recall = {k: [] for k in models}
    for t in range(frames):
        fd = torch.from_numpy(synth.run_frame(3, 0, t)).to(dev)
        last = (t + 1) % 100 == 0
        region = None
        if last:
            region = np.zeros((h, w), bool)
            for cx, cy, a, b in synth.truth(3, 0, t)[0]:
                region |= ((xx - cx) / a) ** 2 + ((yy - cy) / b) ** 2 <= 1.0
        for name, st in streams.items():
            m, _ = st.process(fd, mask=last)
            if last:
                false_fg[name].append(round(float((m[~region] != 0).mean()), 5))
                recall[name].append(round(float((m[region] != 0).mean()), 4))
    for st in streams.values():
        st.close()
    return {"frames": frames, "models": {k: dict(v) for k, v in models.items()},
            "neutral_params": dict(BG_TEST_ONLY),
            "false_foreground_share_every_100_frames": false_fg,
            "hand_recall_every_100_frames": recall}


def bench_single(hmi, synth, torch, dev, cs, args, cfg: int = 2) -> dict:
    """One stream of the given single-stream configuration (640x480 or
    1920x1080): launch shape autotuned for it, pipelined graph-tick
    throughput, the band-test kernel timed alone in plain ticks (its share of
    HBM), and per-frame latency of the synchronous API with a pinned host frame
    (host mask, host pointer)."""
    w, h = synth.shape(cfg)
    st = hmi.Stream(w, h)
    st.learn(torch.from_numpy(synth.learn_frames(cfg)).to(dev))
    ring = [torch.from_numpy(synth.run_frame(cfg, 0, t)).to(dev) for t in range(16)]
    mask = torch.empty((h, w), dtype=torch.uint8, device=dev)
    ptr = torch.zeros(40, dtype=torch.uint8, device=dev)
    b = hmi.hmi_batch_create([st.handle])
    shape, _ = hmi.hmi_batch_autotune(b, [ring[0]], 30, True)

    def tick(k):
        hmi.hmi_batch_process_async(b, [ring[k % 16]], [mask], ptr.data_ptr(), cs.cuda_stream, True)

    def tick_pipelined(k):
        hmi.hmi_batch_process_pipelined(b, [ring[k % 16]], [mask], ptr.data_ptr(), cs.cuda_stream, True)

    for k in range(20):
        tick_pipelined(k)
    hmi.hmi_batch_flush(b, cs.cuda_stream)
    torch.cuda.synchronize()
    steps = max(100, min(args.steps * 4, 4000))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    for k in range(steps):
        tick_pipelined(k)
    hmi.hmi_batch_flush(b, cs.cuda_stream)
    e1.record(cs)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = min(steps, 1000)
    hmi.hmi_batch_profile(b, prof)
    for k in range(prof):
        tick(k)
    ticks, per = hmi.hmi_batch_profile_kernels(b)
    hmi.hmi_batch_profile(b, 0)
    fused = int(shape["fused"])
    cls_ms = per["luma" if fused else "classify"] / max(ticks, 1)
    peak, peak_kind = peaks()
    host = [r.cpu().pin_memory() for r in ring]
    hmask = np.empty((h, w), np.uint8)
    hp = hmi.hmi_pointer()
    lat = []
    for k in range(min(steps, 1000)):
        t = time.perf_counter()
        hmi.hmi_process_frame(st.handle, host[k % 16], hmask, hp)
        lat.append((time.perf_counter() - t) * 1e3)
    hmi.hmi_batch_destroy(b)
    st.close()
    lat.sort()
    bpp = K2_BYTES_PER_PX if fused else CLASSIFY_BYTES_PER_PX
    achieved = bpp * w * h / (cls_ms / 1e3) / 1e9
    return {"frames_per_s": steps / (ms / 1e3), "mpx_per_s": steps * w * h / (ms / 1e3) / 1e6,
            "ms_per_frame": ms / steps, "tuning": shape,
            "launch": "pipelined graph ticks (results one call later), launch shape autotuned for the stream",
            "classify": {"kernel": FUSED_KERNEL[fused] if fused else "k_classify", "launch_us": cls_ms * 1e3,
                         "achieved_GBps": achieved, "frac": achieved / peak,
                         "peak_kind": peak_kind, "bytes_per_px": bpp},
            "k2": k2_roofline(per, ticks, w * h, fused, peak, peak_kind),
            "kernels_us": {k: round(v / max(ticks, 1) * 1e3, 2) for k, v in per.items()},
            "e2e_latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[int(len(lat) * 0.99) - 1],
                               "api": "hmi_process_frame, pinned host frame, host mask + pointer"}}


def bench_serving(hmi, args) -> dict:
    """The 256-stream serving workload: a sweep of arrival rates on short
    traces, served against plain per-frame calls, for the highest frames/s at
    p99 <= 5 ms; then the full-length arrival trace replayed in wall time
    against the server with a device budget below the streams' demand."""
    from paper_1907_04393_gb300 import serve, synth
    n_src = synth.num_streams(serve.CFG)
    bank = serve.FrameBank(range(n_src))
    demand = sum(hmi.hmi_stream_device_bytes(*synth.shape(serve.CFG, i)) for i in range(n_src))
    budget = int(demand * args.serve_budget)
    # the rate sweep first, on fresh servers; then the full-length trace
    rates = [float(x) for x in args.sweep_rates.split(",") if x]
    sweep = None
    if rates and args.sweep_seconds > 0:
        # twice the 256 streams' demand: never reached, so no stream is refused
        sweep = serve.sweep(bank, rates, args.sweep_seconds, budget_bytes=2 * demand)
    tr = serve.make_trace(args.serve_seconds)
    main_run = serve.run_served(tr, bank, budget)
    out = {"workload": "256 streams (128x320x240, 64x640x480, 48x1280x720, 16x1920x1080 RGB8), "
                       "Poisson frame arrivals at 30 fps per stream, Poisson stream joins at 12.8/s, "
                       "exponential lifetimes (mean 20 s), first 30 frames of each stream learned online",
           "trace_s": args.serve_seconds, "streams_in_trace": len(tr.streams),
           "budget_bytes": budget, "demand_bytes_256": demand,
           "latency": "completion (result available on the host) minus scheduled arrival; "
                      "pinned host frames, H2D copy inside",
           **main_run}
    if sweep is not None:
        rows, best = sweep
        keep = ("frames_per_s", "offered_frames_per_s", "p50_ms", "p99_ms", "max_ms",
                "dropped_queue_full", "errors", "frames_per_tick", "round_ms", "saturated",
                "after_first_s", "submit_lag_ms_p99")
        out["sweep"] = [{"rate_scale": r["rate_scale"],
                         "served": {k: r["served"][k] for k in keep if k in r["served"]},
                         "plain": {k: r["plain"][k] for k in keep if k in r["plain"]},
                         "plain_async": {k: r["plain_async"][k] for k in keep + ("cuda_streams",)
                                         if k in r["plain_async"]}} for r in rows]
        out["sweep_trace_s"] = args.sweep_seconds
        out["max_frames_per_s_at_p99_le_5ms"] = best
        out["slo"] = f"p99 <= {serve.SLO_MS} ms, no errors, <= {serve.DROP_BUDGET:.0%} of offered frames dropped"
        out["plain_form"] = "one synchronous hmi_process_frame per frame in arrival order, one thread, " \
                            "streams learned before the trace (no learning work timed)"
        out["plain_async_form"] = "per frame: host-to-device copy, hmi_process_frame_async and a pointer " \
                                  "read-back on one of 8 CUDA streams (stream id mod 8), latency taken by a " \
                                  "completion thread when the frame's event has passed; streams learned up front"
        out["order"] = ("sweep first (the served form at every rate, then the plain forms), "
                        "then the full-length trace")
    return out


def run_serve_only(args) -> None:
    """The serving workload alone (sweep and full-length trace), with nothing
    else run in the process before it."""
    import torch
    from paper_1907_04393_gb300 import hmi
    torch.cuda.set_device(0)
    hmi.load()
    print(json.dumps({"metric": "p99 frame latency and frames/s of the 256-stream serving workload",
                      "serving": bench_serving(hmi, args)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--cpu-ticks", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-single", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-relearn", action="store_true", help="skip the re-learning cost run")
    ap.add_argument("--no-mixture", action="store_true", help="skip the Gaussian mixture run")
    ap.add_argument("--bg-model", choices=sorted(BG_MODELS), default="band",
                    help="background model of every stream of the main workload")
    ap.add_argument("--quality-frames", type=int, default=1200,
                    help="frames of the 1080p drifting scene to compare the background models on (0: skip)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--fused", type=int, choices=[-1, 0, 1, 2], default=-1,
                    help="tick form: 1 the persistent launch, 2 the cooperative per-pixel stage, 0 the "
                         "chain of kernels, -1 the library default (or the autotuner's choice)")
    ap.add_argument("--no-other-form", action="store_true",
                    help="skip timing the other form of the tick")
    ap.add_argument("--mode", choices=["pipelined", "plain"], default="pipelined",
                    help="ticks of the timed region: pipelined (stage overlap) or plain")
    ap.add_argument("--groups", type=int, default=0,
                    help="concurrent stream groups per tick (0: the library default)")
    ap.add_argument("--serve-only", action="store_true",
                    help="only the serving workload, in a fresh process (one JSON line with it)")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-budget", type=float, default=0.9,
                    help="device budget as a fraction of the 256 streams' demand")
    ap.add_argument("--sweep-seconds", type=float, default=5.0)
    ap.add_argument("--sweep-rates", default="1,2,4,8,16")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve_only:
        run_serve_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
