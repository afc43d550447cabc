"""Autotuner for the launch shapes of the rasterizer and the resolve.

Searches the hm_tuning space by timing whole frames of the caller's own
workload with CUDA events: for the direct rasterizer, read-before-atomic
on/off, its register budget and persistent CTAs per SM; the screen-tile
binned rasterizer with its bin (tile) sizes and chunk sizes; and the resolve
tile height.  It keeps the fastest and can cache the choice in a JSON file
keyed by the workload's signature (GPU, resolution, groom count, segments per
frame).  The knobs never change results: visibility is bit-identical and
colours identical under every setting.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

from . import hm


DIRECT = {"raster_bin_w": 0, "raster_bin_h": 0, "raster_bin_chunk": 0}


def candidates():
    out = []
    for pre, mb, th in itertools.product((0, 1), (3, 4), (16, 32)):
        for cps in ((2, 0) if mb == 3 else (2, 3, 0)):
            out.append(dict({"raster_precheck": pre, "raster_min_blocks": mb, "raster_ctas_per_sm": cps,
                             "resolve_tile_h": th}, **DIRECT))
    # the binned rasterizer: bin sizes and chunk sizes (its other knobs fixed)
    for bw, bh, chunk in itertools.product((16, 32), (16, 32), (256, 1024)):
        out.append({"raster_precheck": 0, "raster_min_blocks": 4, "raster_ctas_per_sm": 0, "resolve_tile_h": 32,
                    "raster_bin_w": bw, "raster_bin_h": bh, "raster_bin_chunk": chunk})
    return out


def signature(scene, segments_per_frame: int) -> str:
    import torch
    name = torch.cuda.get_device_name()
    return f"{name}|{scene.camera.width}x{scene.camera.height}|{len(scene.grooms)}|{segments_per_frame}"


def time_frames(step, n: int = 5, warm: int = 2) -> float:
    """Median ms of `step()` (one frame on the current stream)."""
    import torch
    for _ in range(warm):
        step()
    ts = []
    for _ in range(n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def autotune(step, scene=None, segments_per_frame: int = 0, cache_path: str | None = None, n: int = 5,
             verbose: bool = False) -> dict:
    """Pick the fastest tuning for `step` (a frame on the current stream),
    set it with hm.set_tuning and return {"tuning": ..., "ms": ..., "table": [...]}."""
    key = signature(scene, segments_per_frame) if scene is not None else None
    if cache_path and key and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
            if key in cache:
                hm.set_tuning(**cache[key]["tuning"])
                return dict(cache[key], cached=True)
        except (OSError, ValueError):
            pass
    table = []
    for cand in candidates():
        hm.set_tuning(**cand)
        ms = time_frames(step, n=n)
        table.append(dict(cand, ms=ms))
        if verbose:
            print(cand, f"{ms:.4f} ms")
    best = min(table, key=lambda r: r["ms"])
    tuning = {k: best[k] for k in hm.TUNING_FIELDS}
    hm.set_tuning(**tuning)
    res = {"tuning": tuning, "ms": best["ms"], "table": table}
    if cache_path and key:
        cache = {}
        if os.path.exists(cache_path):
            try:
                cache = json.load(open(cache_path))
            except (OSError, ValueError):
                cache = {}
        cache[key] = {"tuning": tuning, "ms": best["ms"]}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
