"""Autotuner of the tiled passes: tile shape and merge schedule.

The labelling passes run on tiles of 32 x TY x TZ sites; the best (TY, TZ)
depends on the lattice sizes, the occupancy and the cluster structure (tile
shape trades shared memory and occupancy against the number of pieces that
cross tile faces).  The merge schedule -- how many unions each lane of the face
merge walks in lockstep (1, 2 or 4), and whether the piece finalize combines the
size additions of the cluster root that collects most of them per warp and CTA --
trades memory-level parallelism against divergence and atomics, and depends on
how many boundary pieces there are and how they cluster.

`tune` times the candidates on the caller's actual batch with CUDA events: every
tile shape at the default schedule, then every schedule at the fastest shape
(results are identical for every candidate; only the time differs).  It keeps
the fastest and caches it in a small JSON file keyed by a signature of the batch
(lattice count, total sites and shape of the largest lattice, each rounded to a
power of two).
"""
from __future__ import annotations

import json
import math
import os

from . import hk

TILES = ((8, 8), (16, 8), (16, 16), (32, 8))
MERGES = ((1, 1), (2, 1), (4, 1), (1, 0), (2, 0), (4, 0))   # (face-merge unions per lane, combine hot root)
DEFAULT_MERGE = (1, 1)   # the library default
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


def _apply(lab, tile, merge):
    lab.set_tile(*tile)
    lab.set_merge(*merge)


def tune(lab: "hk.Labeller", items, stream=None, reps: int = 3, tiles=TILES, merges=MERGES,
         cache: str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """Pick the fastest tile shape and merge schedule for this batch and set them on `lab`.

    Returns {"tile": (ty, tz), "merge": (unions, hot), "ms": {candidate: ms}, "cached": bool}.
    """
    import torch
    sig = signature(items)
    table = _load(cache) if cache else {}
    if not force and sig in table and "merge" in table[sig]:
        best_tile, best_merge = tuple(table[sig]["tile"]), tuple(table[sig]["merge"])
        _apply(lab, best_tile, best_merge)
        return {"tile": best_tile, "merge": best_merge, "ms": table[sig]["ms"], "cached": True}
    stream = stream or torch.cuda.current_stream()
    times = {}

    def time_one(tile, merge):
        _apply(lab, tile, merge)
        with torch.cuda.stream(stream):
            lab.label_batched(items, stream=stream)          # warm-up (sizes the workspace)
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for _ in range(reps):
                lab.label_batched(items, stream=stream)
            end.record(stream)
        end.synchronize()
        ms = start.elapsed_time(end) / reps
        times[f"{tile[0]}x{tile[1]}/u{merge[0]}h{merge[1]}"] = ms
        return ms

    best_tile = min(tiles, key=lambda t: time_one(t, DEFAULT_MERGE))
    best_merge = min(merges, key=lambda m: time_one(best_tile, m) if m != DEFAULT_MERGE else
                     times[f"{best_tile[0]}x{best_tile[1]}/u{m[0]}h{m[1]}"])
    lab.sync_status(stream)
    _apply(lab, best_tile, best_merge)
    if cache:
        table[sig] = {"tile": list(best_tile), "merge": list(best_merge), "ms": times}
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return {"tile": best_tile, "merge": best_merge, "ms": times, "cached": False}
