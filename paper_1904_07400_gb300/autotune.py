"""Autotuner of the persistent batched launch: tries the kernel's tuning knobs (threads per
block, radix preference of the transforms) on a batch, times each with CUDA events on the
current stream, keeps the fastest, and caches the choice in a JSON file keyed by the GPU
name and the batch's grid signature (sizes, orders, precision)."""
from __future__ import annotations

import hashlib
import json
import os

import torch

CANDIDATES = [(512, 0), (512, 1), (256, 0), (256, 1)]


def signature(batch) -> str:
    dims = sorted((p.nx, p.ny, p.order, p.precision) for p in batch.plans)
    h = hashlib.sha1(json.dumps(dims).encode()).hexdigest()[:16]
    return f"{torch.cuda.get_device_name(batch.device)}|n={len(dims)}|{h}"


def _time(batch, reps: int) -> float:
    stream = torch.cuda.current_stream(batch.device)
    batch.launch()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        batch.launch()
    e1.record(stream)
    torch.cuda.synchronize(batch.device)
    return e0.elapsed_time(e1) / reps


def tune(batch, cache_path: str | None = None, reps: int = 5) -> dict:
    """Pick (threads, radix_pref) for `batch`, apply it, and return the record."""
    key = signature(batch)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        rec = cache[key]
        batch.set_config(rec["threads"], rec["radix_pref"])
        return rec
    timings = {}
    for threads, radix in CANDIDATES:
        try:
            batch.set_config(threads, radix)
        except Exception:
            continue
        timings[f"{threads}/{radix}"] = _time(batch, reps)
    best = min(timings, key=timings.get)
    threads, radix = (int(x) for x in best.split("/"))
    batch.set_config(threads, radix)
    rec = {"threads": threads, "radix_pref": radix, "ms": timings[best], "candidates_ms": timings}
    if cache_path:
        cache[key] = rec
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return rec
