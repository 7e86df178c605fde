"""Autotuner of the launch parameters: the tile size (16 or 32 pixels, a
property of the step's batch), and through gs_set_tuning the splat records
staged per round by the compositing forward and by its backward, and the
grid (blocks per SM) of the sort's grid-stride kernels.  Every candidate
gives the same images and gradients (the parameters change only how work is
split).  The tuner runs the caller's own joint step: per tile size, the two
staging batches are chosen from the forward's and the backward's own stage
times, then the sort grid from the whole step's time; the tile size with the
fastest step wins.  The result is cached per (GPU, SM count, workload
shape)."""
from __future__ import annotations

import json
import os

import torch

from .core import TileLists, gs_get_tuning, gs_set_tuning

# the usual winner last, so that the step is left as it was tried (no
# rebuild of the batch buffers after the trials)
TILES = (32, 16)
RENDER_BATCHES = (64, 128, 256)
SORT_BLOCKS = (1, 2, 4)
# (render_fwd_batch, render_bwd_batch, sort_blocks_per_sm) settings the
# tuner tries; all must give identical results
CANDIDATES = [(rb, rb, 2) for rb in RENDER_BATCHES] + [(256, 128, sb) for sb in SORT_BLOCKS]


def _cache_path():
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_2603_04847_gb300", "autotune.json")


def _key(js) -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    g = js.g
    return "%s|%d|N=%d|K=%d|B=%d|P=%d|%s" % (
        p.name, p.multi_processor_count, g.n, g.sh.shape[1], js.batch.B, js.batch.n_pixels, js.mode)


def _realloc(js):
    """Re-create the sort workspaces and drop the captured graph, whose
    launches carry the old grids."""
    for r in js.renderers:
        r.tl = TileLists(r.n, r.batch, r.tl.capacity, r.image.device)
    js.graph = None


def _median(xs):
    xs = sorted(xs)
    return xs[len(xs) // 2]


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
    return _median(times)


def _time_stages(js, reps: int, names=("render_fwd", "raster_bwd")) -> dict:
    """Median device time (ms) of the named stages of the step."""
    st = torch.cuda.current_stream()
    js.step()
    acc = {n: [] for n in names}
    for _ in range(reps):
        marks = []

        def mark(name):
            e = torch.cuda.Event(enable_timing=True)
            e.record(st)
            marks.append((name, e))

        first = torch.cuda.Event(enable_timing=True)
        first.record(st)
        js.step(mark)
        torch.cuda.synchronize()
        tot = {n: 0.0 for n in names}
        prev = first
        for name, e in marks:
            if name in tot:
                tot[name] += prev.elapsed_time(e)
            prev = e
        for n in names:
            acc[n].append(tot[n])
    return {n: _median(v) for n, v in acc.items()}


def _set(rf, rb, sb, js):
    gs_set_tuning(rf, rb, sb)
    _realloc(js)


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
        js.set_tile(t["tile"])
        _set(t["render_fwd_batch"], t["render_bwd_batch"], t["sort_blocks_per_sm"], js)
        js.ensure_capacity()
        return dict(t, cached=True)
    timings = {}
    sb0 = gs_get_tuning()["sort_blocks_per_sm"]
    per_tile = {}
    for tile in TILES:
        js.set_tile(tile)
        js.ensure_capacity()
        stage = {}
        for rb in RENDER_BATCHES:
            _set(rb, rb, sb0, js)
            stage[rb] = _time_stages(js, reps)
            timings["tile%d/stages@%d" % (tile, rb)] = stage[rb]
        rf = min(RENDER_BATCHES, key=lambda r: stage[r]["render_fwd"])
        rbw = min(RENDER_BATCHES, key=lambda r: stage[r]["raster_bwd"])
        step_ms = {}
        for sb in SORT_BLOCKS:
            _set(rf, rbw, sb, js)
            step_ms[sb] = _time_step(js, reps)
            timings["tile%d/step@sort%d" % (tile, sb)] = step_ms[sb]
        sb = min(SORT_BLOCKS, key=step_ms.get)
        per_tile[tile] = dict(tile=tile, render_fwd_batch=rf, render_bwd_batch=rbw, sort_blocks_per_sm=sb,
                              ms=step_ms[sb])
    best = min(per_tile.values(), key=lambda t: t["ms"])
    js.set_tile(best["tile"])
    _set(best["render_fwd_batch"], best["render_bwd_batch"], best["sort_blocks_per_sm"], js)
    js.ensure_capacity()
    if use_cache:
        cache[key] = best
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return dict(best, timings=timings, cached=False)
