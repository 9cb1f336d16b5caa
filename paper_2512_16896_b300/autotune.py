"""Launch-shape autotuner for the persistent collision kernel.

Times sc_collide_ex over a grid of launch shapes (threads per CTA, A spheres
per lane, B-segment length, CTAs per SM) on a bounded sample of the batch's
candidates (kept in the batch's LPT order, so the sample has the batch's mix
of heavy and light candidates), and returns the fastest. Results are cached in
a JSON file keyed by the device name and a histogram of the batch's per-template
sphere counts, so a workload of the same shape reuses the choice.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np
import torch

from . import _native as nat

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")

DEFAULT_SPACE = [
    (t, apl, seg, cps)
    for apl, ts in ((2, (256, 512)), (4, (128, 256, 512)))
    for t in ts
    for seg in (128, 256, 512)
    for cps in (1, 2, 4)
]


def shape_key(batch, first_new: int) -> str:
    nsph = np.asarray(batch.obj_sph_off[np.asarray(batch.tmpl_obj_off)[1:]] -
                      batch.obj_sph_off[np.asarray(batch.tmpl_obj_off)[:-1]])
    nobj = np.diff(batch.tmpl_obj_off)
    h = np.histogram(nsph, bins=[0, 64, 256, 1024, 2048, 4096, 8193])[0]
    o = np.histogram(nobj, bins=[0, 4, 8, 16, 32, 64, 257])[0]
    nobb = int(len(batch.obb))
    frac = lambda x: tuple(np.round(x / max(1, x.sum()), 2).tolist())
    raw = json.dumps([frac(h), frac(o), nobb > 0, first_new > 0])
    return hashlib.sha1(raw.encode()).hexdigest()[:16]


def _load():
    if os.path.exists(CACHE):
        try:
            return json.load(open(CACHE))
        except (OSError, ValueError):
            return {}
    return {}


def tune_collide(ctx: nat.Context, db: nat.DeviceBatch, batch, poses: torch.Tensor, order: torch.Tensor,
                 first_new: int = 0, space=None, sample: int = 16384, reps: int = 2, use_cache: bool = True,
                 verbose: bool = False):
    """Best (threads, a_per_lane, seg_len, ctas_per_sm) for this batch shape."""
    dev = torch.cuda.get_device_name(ctx.device)
    key = f"{dev}|{shape_key(batch, first_new)}"
    cache = _load()
    if use_cache and key in cache:
        return tuple(cache[key]["config"]), cache[key]
    space = space or DEFAULT_SPACE
    n = order.numel()
    if n > sample:  # evenly strided sample of the LPT list keeps its work profile
        idx = torch.linspace(0, n - 1, sample, device=order.device).long()
        sub = order[idx].contiguous()
    else:
        sub = order
    results = []
    for cfg in space:
        try:
            nat.collide(ctx, db, poses, active=sub, first_new=first_new, config=cfg)  # warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            for _ in range(reps):
                nat.collide(ctx, db, poses, active=sub, first_new=first_new, config=cfg)
            e1.record(ctx.stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
        except nat.SceniError:
            continue  # shape not launchable for this batch (e.g. shared memory)
        results.append((ms, cfg))
        if verbose:
            print(f"  {cfg}: {ms:.3f} ms", flush=True)
    results.sort()
    best_ms, best = results[0]
    entry = {"config": list(best), "ms": best_ms, "sample": int(sub.numel()),
             "top": [[round(m, 4), list(c)] for m, c in results[:8]], "when": time.strftime("%Y-%m-%d %H:%M:%S")}
    cache[key] = entry
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return best, entry
