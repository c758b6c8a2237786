"""Launch-shape cache for batches (Sec. 3.3: the GPU computation is autotuned).

The search itself runs in the library (hmi_batch_autotune times candidate
launch shapes with CUDA events).  This module keeps its results in a JSON file
keyed by the GPU model, the tick form (pipelined or plain) and the multiset
of frame shapes of the batch, so that a batch with a known key gets its launch
shape without searching again.
"""
from __future__ import annotations

import json
import os

from . import hmi

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hmi_gb300_autotune.json")


def key(gpu_name: str, shapes, pipelined: bool) -> str:
    mix = ",".join(f"{w}x{h}" for w, h in sorted(shapes))
    return f"{gpu_name}|{'pipelined' if pipelined else 'plain'}|{mix}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(batch: int, shapes, frames, gpu_name: str, pipelined: bool = True, ticks: int = 50,
         cache_path: str | None = DEFAULT_CACHE) -> dict:
    """Apply the cached launch shape for this key, or search one and cache it.
    frames: one device frame per stream of the batch (used only on a miss).
    Returns {"tuning": ..., "tick_us": ..., "cached": bool, "key": ...}."""
    k = key(gpu_name, shapes, pipelined)
    cache = _load(cache_path) if cache_path else {}
    hit = cache.get(k)
    if hit is not None:
        try:
            hmi.hmi_batch_set_tuning(batch, hit["tuning"])
            return {**hit, "cached": True, "key": k}
        except (hmi.HmiError, KeyError, TypeError):
            pass                      # stale or malformed entry: search again
    tuning, us = hmi.hmi_batch_autotune(batch, frames, ticks, pipelined)
    entry = {"tuning": tuning, "tick_us": us}
    if cache_path:
        cache[k] = entry
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        tmp = f"{cache_path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return {**entry, "cached": False, "key": k}
