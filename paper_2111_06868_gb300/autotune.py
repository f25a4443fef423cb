"""Project-written autotuner for batched runs: picks the shared-memory tile
shape (tile_bits, max_high) and CTAs per SM by timing candidate plans of the
actual batch on the device, and caches the winner per (device, batch
signature) in a JSON file."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import hq

CANDIDATES = [(12, 6, 0, 0), (13, 7, 0, 0), (13, 6, 0, 0), (11, 5, 0, 0), (13, 7, 0, 1), (12, 6, 0, 1)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hq_gb300", "autotune.json")


def signature(circuits) -> str:
    h = hashlib.sha1()
    for c in circuits:
        h.update(f"{c.n}:{len(c.gates)};".encode())
    return h.hexdigest()[:16]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(circuits, states=None, candidates=CANDIDATES, reps: int = 3, cache_path: str | None = DEFAULT_CACHE,
         objective: str = "makespan"):
    """Returns (tile_bits, max_high, ctas_per_sm, small_first, timings) with the
    best score -- median makespan, or median per-circuit latency when
    objective="p50" -- reusing the cached choice when the signature matches."""
    import torch

    dev = torch.cuda.get_device_name()
    key = f"{dev}|{signature(circuits)}|{objective}"
    if cache_path:
        cached = _load(cache_path).get(key)
        if cached:
            return tuple(cached["choice"]) + (cached.get("timings", {}),)
    candidates = [tuple(c) + (0,) * (4 - len(c)) for c in candidates]
    timings = {}
    for cand in candidates:
        b = hq.Batch(circuits, states, *cand)
        b.run()
        spans = []
        for _ in range(reps):
            b.run()
            lat, span = b.latencies()
            spans.append(float(np.percentile(lat, 50)) if objective == "p50" else span)
        b.close()
        timings[str(cand)] = sorted(spans)[len(spans) // 2]
    best = min(candidates, key=lambda c: timings[str(c)])
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        data = _load(cache_path)
        data[key] = {"choice": list(best), "timings": timings}
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1)
    return tuple(best) + (timings,)
