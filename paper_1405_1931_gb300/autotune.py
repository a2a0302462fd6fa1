"""Tile-shape autotuner.

The labelling passes run on tiles of 32 x TY x TZ sites; the best (TY, TZ)
depends on the lattice sizes, the occupancy and the cluster structure (tile
shape trades shared memory and occupancy against the number of pieces that
cross tile faces).  `tune` times every supported shape on the caller's actual
batch with CUDA events and keeps the fastest; results are cached in a small
JSON file keyed by a signature of the batch (lattice count, total sites and
shape of the largest lattice, each rounded to a power of two).
"""
from __future__ import annotations

import json
import math
import os

from . import hk

TILES = ((8, 8), (16, 8), (16, 16), (32, 8))
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hk_autotune.json")


def signature(items) -> str:
    """items: list of (phi, periodic, out) as taken by Labeller.label_batched."""
    sites = sum(int(phi.numel()) for phi, _, _ in items)
    biggest = max(items, key=lambda it: it[0].numel())[0].shape
    r = lambda v: 1 << max(0, int(math.log2(max(int(v), 1))))
    return f"n{r(len(items))}_s{r(sites)}_b{r(biggest[2])}x{r(biggest[1])}x{r(biggest[0])}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(lab: "hk.Labeller", items, stream=None, reps: int = 3, tiles=TILES, cache: str | None = DEFAULT_CACHE,
         force: bool = False) -> dict:
    """Pick the fastest tile shape for this batch and set it on `lab`.

    Returns {"tile": (ty, tz), "ms": {shape: ms}, "cached": bool}.
    """
    import torch
    sig = signature(items)
    table = _load(cache) if cache else {}
    if not force and sig in table:
        best = tuple(table[sig]["tile"])
        lab.set_tile(*best)
        return {"tile": best, "ms": table[sig]["ms"], "cached": True}
    stream = stream or torch.cuda.current_stream()
    times = {}
    for tile in tiles:
        lab.set_tile(*tile)
        with torch.cuda.stream(stream):
            lab.label_batched(items, stream=stream)          # warm-up (sizes the workspace)
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for _ in range(reps):
                lab.label_batched(items, stream=stream)
            end.record(stream)
        end.synchronize()
        times[f"{tile[0]}x{tile[1]}"] = start.elapsed_time(end) / reps
    best_key = min(times, key=times.get)
    best = tuple(int(v) for v in best_key.split("x"))
    lab.set_tile(*best)
    if cache:
        table[sig] = {"tile": list(best), "ms": times}
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return {"tile": best, "ms": times, "cached": False}
