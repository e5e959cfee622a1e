"""Tile-shape autotuner for the fused fine-tile kernel.

For a problem (or batch) it times a few optimiser steps with each candidate
tile shape, with and without the persistent launch, picks the fastest and
remembers it in a JSON cache keyed by the problem's signature (PDE, dtype,
level shapes of every instance).  Timing uses CUDA events on the problem's
stream; the measurement function can be replaced (tests use a fake one).
"""
from __future__ import annotations

import hashlib
import json
import os

ST_TILES = ((16, 32), (16, 64), (8, 64), (32, 32), (8, 128))
STREAM_TILE = (32, 60)   # Burgers: the warp-streaming kernel's strip (no persistent variant)
NS2D_TILES = ((8, 32), (16, 32))
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "modil_gb300", "autotune.json")


def signature(descs):
    """Stable key of a batch: PDE, dtype, and every instance's grid and levels."""
    h = hashlib.sha256()
    for d in descs:
        h.update(repr((d.pde, d.dtype, d.shape, d.n_levels)).encode())
    return f"pde{descs[0].pde}-dt{descs[0].dtype}-n{len(descs)}-{h.hexdigest()[:16]}"


def time_steps(descs, tile, persistent, steps=20, warmup=5):
    """Milliseconds per optimiser step of the batch with the given tile shape."""
    import torch

    from . import modil
    ds = [modil.Desc(**{**d.kwargs, "tile": tile}) for d in descs]
    with modil.Problem(ds) as p:
        if persistent:
            p.set_persistent(True)
        p.step(warmup, read_loss=False)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(p.stream)
        p.step(steps, read_loss=False)
        b.record(p.stream)
        b.synchronize()
        return a.elapsed_time(b) / steps


def autotune(descs, candidates=None, persistent_options=(False, True), measure=time_steps,
             cache_path=DEFAULT_CACHE, use_cache=True):
    """Best (tile, persistent, ms_per_step) for the batch; cached by signature."""
    key = signature(descs)
    cache = {}
    if use_cache and cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            c = cache[key]
            return tuple(c["tile"]), bool(c["persistent"]), float(c["ms"])
    if candidates is None:
        candidates = NS2D_TILES if descs[0].pde == 3 else ST_TILES
        if descs[0].pde == 1 and not any(d._pts is not None for d in descs):
            candidates = candidates + (STREAM_TILE,)
    best = None
    results = []
    for tile in candidates:
        for pers in persistent_options:
            if pers and (descs[0].pde == 3 or tuple(tile) == STREAM_TILE):
                continue
            ms = float(measure(descs, tile, pers))
            results.append((tile, pers, ms))
            if best is None or ms < best[2]:
                best = (tuple(tile), bool(pers), ms)
    if cache_path:
        cache[key] = {"tile": list(best[0]), "persistent": best[1], "ms": best[2],
                      "tried": [[list(t), p, m] for t, p, m in results]}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best
