"""Autotuner of the batched halo paste: tile shape, work-unit size (halos per unit,
the "bin capacity") and persistent CTAs per SM, timed on the device with CUDA events on
the workload itself; results cached as JSON keyed by a workload signature."""
from __future__ import annotations

import hashlib
import json
import os

import torch

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "bp_gb300", "autotune.json")


def _signature(n, g, ap_r500, extra=""):
    s = f"hp:{n}:{g.nx}x{g.ny}x{g.n_maps}:{g.dtheta:.6e}:{ap_r500}:{extra}"
    return hashlib.sha256(s.encode()).hexdigest()[:16]


def tune_hp(ctx, thx, thy, vlos, model, status, g, maps, ap_r500=0.0, map_id=None,
            tiles=(32, 64), units=(0, 256, 1024, 4096), ctas=(0, 1, 2), reps=3,
            cache_path=DEFAULT_CACHE, use_cache=True, tag=""):
    """Times every (tile, unit, ctas_per_sm) on this catalogue and returns
    {"tile", "unit", "ctas_per_sm", "ms", "trials"}."""
    key = _signature(thx.numel(), g, ap_r500, tag)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True)
    trials = []
    for tile in tiles:
        for unit in units:
            for cps in ctas:
                plan = ctx.hp_plan(thx, thy, model, status, g, ap_r500, map_id, tile, unit, cps)
                maps.zero_()
                plan.execute(thx, thy, vlos, model, status, maps, map_id)  # warm-up
                times = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    plan.execute(thx, thy, vlos, model, status, maps, map_id)
                    e1.record()
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                plan.close()
                trials.append({"tile": tile, "unit": unit, "ctas_per_sm": cps,
                               "ms": min(times)})
    best = min(trials, key=lambda t: t["ms"])
    out = dict(best, trials=trials)
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache[key] = out
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return dict(out, cached=False)
