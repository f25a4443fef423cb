"""Project-written autotuner for batched runs: picks the in-pass fusion width
(Sec. 3.1 compress into blocks of at most fuse_k = 1, 2 or 3 qubits), the
shared-memory tile shape (tile_bits, max_high) and CTAs per SM by timing
candidate plans of the actual batch on the device, and caches the winner per
(device, batch signature, objective) in a JSON file.

A candidate is (tile_bits, max_high, ctas_per_sm, small_first, fuse_k); the
search is the cross product of TILES and FUSE_WIDTHS, each timed as the
median of `reps` graph replays."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import hq

TILES = [(12, 6, 0), (13, 7, 0), (13, 6, 0), (11, 5, 0)]
FUSE_WIDTHS = [1, 2, 3]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hq_gb300", "autotune.json")


def candidates(small_first: int = 0, tiles=TILES, widths=FUSE_WIDTHS):
    return [(t, h, c, small_first, k) for (t, h, c) in tiles for k in widths]


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


def tune(circuits, states=None, cands=None, reps: int = 3, cache_path: str | None = DEFAULT_CACHE,
         objective: str = "makespan", small_first: int = 0):
    """Returns (choice, timings): choice = (tile_bits, max_high, ctas_per_sm,
    small_first, fuse_k) with the best score -- median makespan, or median
    per-circuit latency when objective="p50" -- reusing the cached choice when
    the signature matches; timings maps each candidate to its score (s)."""
    import torch

    dev = torch.cuda.get_device_name()
    key = f"{dev}|{signature(circuits)}|{objective}|{small_first}"
    if cache_path:
        cached = _load(cache_path).get(key)
        if cached:
            return tuple(cached["choice"]), cached.get("timings", {})
    cands = [tuple(c) + (0,) * (5 - len(c)) for c in (cands or candidates(small_first))]
    timings = {}
    for cand in cands:
        b = hq.Batch(circuits, states, *cand)
        b.run()
        scores = []
        for _ in range(reps):
            b.run()
            lat, span = b.latencies()
            scores.append(float(np.percentile(lat, 50)) if objective == "p50" else span)
        b.close()
        timings[str(cand)] = sorted(scores)[len(scores) // 2] * 1e-6
    best = min(cands, key=lambda c: timings[str(c)])
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        data = _load(cache_path)
        data[key] = {"choice": list(best), "timings": timings}
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1)
    return tuple(best), timings
