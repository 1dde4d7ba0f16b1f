"""Autotuner of the batched launch: tries the persistent kernels (the one on the transform
network's item bodies, and the generic one with its threads per block and radix preference
of the transforms) and the streams form (each grid's own kernels on 2,
4, 8 or 16 internal streams) on a batch, times each with CUDA events on the current stream,
keeps the fastest, and caches the choice in a JSON file keyed by the GPU name and the
batch's grid signature (sizes, orders, precision)."""
from __future__ import annotations

import hashlib
import json
import os

import torch

# (threads, second knob): 64 is the persistent kernel on the network's item bodies with 1, 2,
# 4 or 8 units per item; 256 and 512 the generic one with radix 8 (0) or radix 4 (1) first
CANDIDATES = [(64, 1), (64, 2), (64, 4), (64, 8), (64, 16), (512, 0), (512, 1), (256, 0), (256, 1)]
STREAMS = (2, 4, 8, 16)


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


def _apply(batch, rec: dict) -> None:
    if rec.get("mode") == "streams":
        batch.set_streams(rec["streams"])
    else:
        batch.set_config(rec["threads"], rec["radix_pref"])


def tune(batch, cache_path: str | None = None, reps: int = 5) -> dict:
    """Pick the batch's form and knobs, apply them, and return the record."""
    key = signature(batch)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        rec = cache[key]
        _apply(batch, rec)
        return rec
    timings, recs = {}, {}
    for threads, radix in CANDIDATES:
        rec = {"mode": "persistent", "threads": threads, "radix_pref": radix}
        try:
            _apply(batch, rec)
        except Exception:
            continue
        name = f"{threads}/{radix}"
        timings[name], recs[name] = _time(batch, reps), rec
    for n in STREAMS:
        rec = {"mode": "streams", "streams": n}
        _apply(batch, rec)
        name = f"streams/{n}"
        timings[name], recs[name] = _time(batch, reps), rec
    best = min(timings, key=timings.get)
    rec = dict(recs[best], ms=timings[best], candidates_ms=timings)
    _apply(batch, rec)
    if cache_path:
        cache[key] = rec
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return rec
