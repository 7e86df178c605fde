"""Autotuner of the launch parameters (gs_set_tuning): splat records staged
per round by the compositing kernels, and the grid (blocks per SM) of the
sort's grid-stride kernels.  Every candidate gives the same result (the parameters change only
how work is split); the tuner times the caller's own joint step under each
and keeps the fastest, cached per (GPU, SM count, workload shape)."""
from __future__ import annotations

import json
import os

import torch

from .core import TileLists, gs_get_tuning, gs_set_tuning

CANDIDATES = [(rb, sb) for rb in (64, 128, 256) for sb in (1, 2, 4)]


def _cache_path():
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_2603_04847_gb300", "autotune.json")


def _key(js) -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    g = js.g
    return "%s|%d|N=%d|K=%d|B=%d|P=%d|tiles=%d|%s" % (
        p.name, p.multi_processor_count, g.n, g.sh.shape[1], js.batch.B, js.batch.n_pixels, js.batch.n_tiles,
        js.mode)


def _realloc(js):
    """Re-create the sort workspaces and drop the captured graph, whose
    launches carry the old grids."""
    for r in js.renderers:
        r.tl = TileLists(r.n, r.batch, r.tl.capacity, r.image.device)
    js.graph = None


def _time_step(js, reps: int) -> float:
    st = torch.cuda.current_stream()
    js.step()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        js.step()
        b.record(st)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def autotune(js, reps: int = 5, use_cache: bool = True, cache_path: str = None) -> dict:
    """Sets the fastest tuning for the JointStep `js` (whose parameters it
    advances by a few optimiser steps) and returns it with the timings."""
    cache_path = cache_path or _cache_path()
    key = _key(js)
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        t = cache[key]
        gs_set_tuning(t["render_batch"], t["sort_blocks_per_sm"])
        _realloc(js)
        return dict(t, cached=True)
    timings = {}
    for rb, sb in CANDIDATES:
        gs_set_tuning(rb, sb)
        _realloc(js)
        timings["%d/%d" % (rb, sb)] = _time_step(js, reps)
    best = min(timings, key=timings.get)
    rb, sb = (int(x) for x in best.split("/"))
    gs_set_tuning(rb, sb)
    _realloc(js)
    result = dict(render_batch=rb, sort_blocks_per_sm=sb, ms=timings[best], timings=timings)
    if use_cache:
        cache[key] = dict(render_batch=rb, sort_blocks_per_sm=sb, ms=timings[best])
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return dict(result, cached=False)


def current() -> dict:
    return gs_get_tuning()
