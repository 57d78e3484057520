"""Autotuner for the batched form.

Times candidate settings of the batch knobs (table load bound, contraction
block size, points per thread, warp pre-aggregation) on a deterministic sample
of the instances and keeps the fastest.  The knobs never change results (each
table is sized so that it cannot overflow), only speed.  Choices are cached in
a JSON file keyed by GPU name and a signature of the workload.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from .batch import RasterBatch

DEFAULT = {"load": 0.75, "block": 256, "width": 4, "preagg": 1}
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")


def _signature(instances) -> str:
    h = hashlib.sha1()
    for xy, p, tau, mu in instances:
        h.update(f"{xy.shape[0]}:{p}:{tau}:{mu};".encode())
    return h.hexdigest()[:16]


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(c: dict):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time(instances, cfg, reps: int) -> float:
    b = RasterBatch(instances, **cfg)
    try:
        b.run()
        b.wait(allow_range_error=True)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            b.run()
        e.record()
        b.wait(allow_range_error=True)
        return s.elapsed_time(e) / reps
    finally:
        b.close()
        torch.cuda.synchronize()


def candidates():
    out = []
    for load in (0.5, 0.75):
        for width in (2, 4, 8):
            for preagg in (0, 1):
                out.append({"load": load, "block": 256, "width": width, "preagg": preagg})
    return out


def tune_batch(instances, sample: int = 256, reps: int = 3, use_cache: bool = True, log=None) -> dict:
    """Best knob setting for these instances (list of (xy, precision, tau, mu))."""
    gpu = torch.cuda.get_device_name()
    sig = _signature(instances)
    key = f"{gpu}|{sig}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return dict(cache[key]["config"])
    step = max(1, len(instances) // sample)
    sub = instances[::step][:sample]
    results = []
    for cfg in candidates():
        results.append((_time(sub, cfg, reps), cfg))
    best_t, best = min(results, key=lambda r: r[0])
    for block in (128, 512):  # then the block size around the best setting
        cfg = dict(best, block=block)
        t = _time(sub, cfg, reps)
        results.append((t, cfg))
        if t < best_t:
            best_t, best = t, cfg
    if log is not None:
        log.extend({"ms": t, **c} for t, c in results)
    cache[key] = {"config": best, "ms": best_t, "sample": len(sub)}
    if use_cache:
        _store_cache(cache)
    return dict(best)
