"""Autotuner for the blend launch configuration: tile shape, shared-memory batch size and pixels
per thread of the forward and of the backward blend.

Every candidate renders the same frame (forward + backward) a few times; the fastest one wins
and is cached in a JSON file keyed by the workload's signature (view sizes, Gaussian count
bucket, SH degree). Per-pixel results do not depend on these choices (the rasterizer's blend is
independent of tiling, batching and pixels per thread), so the tuner only trades speed.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import replace

import torch

from .rasterizer import Rasterizer, RenderSettings

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "odgs_autotune.json")

TILES = ((16, 16), (16, 8), (32, 8), (8, 8), (32, 16), (16, 32))
BATCHES = (32, 64, 128)
PPTS = (4, 2)


def valid(tile_w: int, tile_h: int, ppt: int, widths) -> bool:
    """Mirror of the library's checks: W divisible by tile_w, whole warps, at most 256 threads."""
    area = tile_w * tile_h
    if tile_w not in (8, 16, 32) or area < 32 or area > 1024 or area % 32:
        return False
    if tile_w % ppt or (area // ppt) % 32 or area // ppt > 256:
        return False
    return all(w % tile_w == 0 for w in widths)


def candidates(widths, tiles=TILES, batches=BATCHES, ppts=PPTS):
    """(tile_w, tile_h, batch, forward pixels per thread, backward pixels per thread)."""
    out = []
    for (tw, th) in tiles:
        for pf in ppts:
            for pb in ppts:
                if not (valid(tw, th, pf, widths) and valid(tw, th, pb, widths)):
                    continue
                for b in batches:
                    out.append((tw, th, b, pf, pb))
    return out


def signature(n: int, views, sh_degree: int) -> str:
    sizes = ",".join(f"{v.width}x{v.height}" for v in views)
    bucket = 2 ** int(round(math.log2(max(n, 1))))
    return f"n~{bucket}|sh{sh_degree}|{sizes}"


def _time_frame(rast, params, views, rs, grads, iters):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    imgs, _ = rast.forward(*params, views, rs, want_T=False)  # also sizes the buffers
    gi = [torch.ones_like(im) / im.numel() for im in imgs]
    rast.backward(gi, grads)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(iters):
        rast.forward(*params, views, rs, want_T=False)
        rast.backward(gi, grads)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / iters


def autotune(params, views, base: RenderSettings = None, cache_path: str = DEFAULT_CACHE, iters: int = 3,
             cands=None, use_cache: bool = True, verbose: bool = False) -> RenderSettings:
    """Fastest (tile_w, tile_h, batch, pixels per thread forward / backward) for this frame, from the
    cache when known."""
    base = base or RenderSettings()
    key = signature(params[0].shape[0], views, base.sh_degree)
    cache = {}
    if use_cache and cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        c = cache[key]
        return replace(base, tile_w=c["tile_w"], tile_h=c["tile_h"], batch=c["batch"], pixels_per_thread=c["ppt"],
                       pixels_per_thread_bwd=c.get("ppt_bwd", c["ppt"]))
    cands = cands or candidates([v.width for v in views])
    rast = Rasterizer(params[0].device, capacity_mode="query")
    grads = {k: torch.empty_like(t) for k, t in zip(("means", "scales", "quats", "opacity", "sh"), params)}
    best, best_ms, results = None, float("inf"), []
    for (tw, th, b, pf, pb) in cands:
        rs = replace(base, tile_w=tw, tile_h=th, batch=b, pixels_per_thread=pf, pixels_per_thread_bwd=pb)
        ms = _time_frame(rast, params, views, rs, grads, iters)
        results.append({"tile_w": tw, "tile_h": th, "batch": b, "ppt": pf, "ppt_bwd": pb, "ms": ms})
        if verbose:
            print(f"autotune {tw}x{th} batch {b} ppt {pf}/{pb}: {ms:.3f} ms", flush=True)
        if ms < best_ms:
            best, best_ms = (tw, th, b, pf, pb), ms
    tw, th, b, pf, pb = best
    if cache_path:
        cache[key] = {"tile_w": tw, "tile_h": th, "batch": b, "ppt": pf, "ppt_bwd": pb, "ms": best_ms,
                      "tried": len(results)}
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return replace(base, tile_w=tw, tile_h=th, batch=b, pixels_per_thread=pf, pixels_per_thread_bwd=pb)
