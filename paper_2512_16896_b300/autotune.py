"""Launch-shape autotuner for the persistent collision kernel and the
generation kernels.

tune_collide times sc_collide_ex over a grid of launch shapes (threads per
CTA, A spheres per lane, B-segment length, CTAs per SM) on a bounded sample
of the batch's candidates (kept in the batch's LPT order, so the sample has
the batch's mix of heavy and light candidates). tune_generate times whole
sc_generate calls (CUDA-graph replays, the reachability stage included when
an arm is given) over the generation kernels' shapes (threads per CTA, A
spheres per lane, CTAs per SM). Each returns the fastest shape. Results are
cached in a JSON file keyed by the device name, the call and histograms of the
batch's per-template sphere and object counts, so a workload of the same
shape reuses the choice. Every shape computes the same results (the launch
shape changes only how the work is spread), which the tests check.
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


GENERATE_SPACE = [
    (t, apl, 256, cps)
    for t in (128, 256)
    for apl in (1, 2)
    for cps in (2, 3, 4, 6)
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


def generate_key(batch, retries: int, reach: bool, gated: bool) -> str:
    return f"generate|{shape_key(batch, 0)}|r{retries}|{'reach' if reach else 'plain'}|{'gate' if gated else 'nogate'}"


def _load():
    if os.path.exists(CACHE):
        try:
            return json.load(open(CACHE))
        except (OSError, ValueError):
            return {}
    return {}


def tune_collide(ctx: nat.Context, db: nat.DeviceBatch, batch, poses: torch.Tensor, order: torch.Tensor,
                 first_new: int = 0, space=None, sample: int = 16384, reps: int = 2, use_cache: bool = True,
                 verbose: bool = False, decide: bool = False):
    """Best launch configuration for this batch shape, in exact-minimum mode
    or (decide) decide-only mode: the fastest (threads, a_per_lane, seg_len,
    ctas_per_sm) of the space, then that shape with the local spheres staged
    by per-lane loads or by one bulk copy, whichever is faster. Returns the
    full sc_collide_config tuple (threads, a_per_lane, seg_len, ctas_per_sm,
    decide_only, stage_bulk) and the cache entry."""
    dev = torch.cuda.get_device_name(ctx.device)
    key = f"{dev}|{shape_key(batch, first_new)}|{'decide' if decide else 'exact'}"
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
    mode = 1 if decide else 0

    def time_cfg(full):
        nat.collide(ctx, db, poses, active=sub, first_new=first_new, config=full)  # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(reps):
            nat.collide(ctx, db, poses, active=sub, first_new=first_new, config=full)
        e1.record(ctx.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    results = []
    for cfg in space:
        full = tuple(cfg)[:4] + (mode, 0)
        try:
            ms = time_cfg(full)
        except nat.SceniError:
            continue  # shape not launchable for this batch (e.g. shared memory)
        results.append((ms, full))
        if verbose:
            print(f"  {full}: {ms:.3f} ms", flush=True)
    if results:
        best = min(results)[1]
        bulk = best[:5] + (1,)
        try:
            ms = time_cfg(bulk)
            results.append((ms, bulk))
            if verbose:
                print(f"  {bulk}: {ms:.3f} ms", flush=True)
        except nat.SceniError:
            pass
    return _store(cache, key, results, int(sub.numel()))


def _store(cache, key, results, sample):
    if not results:
        raise nat.SceniError("no launch shape of the search space could run this batch")
    results.sort()
    best_ms, best = results[0]
    entry = {"config": list(best), "ms": best_ms, "sample": sample,
             "top": [[round(m, 4), list(c)] for m, c in results[:8]], "when": time.strftime("%Y-%m-%d %H:%M:%S")}
    cache[key] = entry
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return tuple(best), entry


def tune_generate(ctx: nat.Context, db: nat.DeviceBatch, batch, order: torch.Tensor, seed: int = 1,
                  max_retries: int = 10, arm=None, ik=None, gate=None, space=None, reps: int = 2,
                  use_cache: bool = True, verbose: bool = False):
    """Best (threads, a_per_lane, seg_len, ctas_per_sm) of sc_generate for this
    batch shape: each shape's call is captured once into a CUDA graph, warmed
    and replayed `reps` times on the whole batch (the generation kernels'
    balance depends on the whole candidate list, so no sample is taken)."""
    dev = torch.cuda.get_device_name(ctx.device)
    key = f"{dev}|{generate_key(batch, max_retries, arm is not None, gate is not None)}"
    cache = _load()
    if use_cache and key in cache:
        return tuple(cache[key]["config"]), cache[key]
    space = space or GENERATE_SPACE
    poses = db.new_poses(order.device)
    n = db.n_cand
    outs = (torch.zeros(n, dtype=torch.uint8, device=poses.device), torch.zeros(n, dtype=torch.uint8, device=poses.device),
            torch.zeros(n, dtype=torch.int32, device=poses.device))
    results = []
    for cfg in space:
        try:
            call = lambda: nat.generate(ctx, db, seed=seed, max_retries=max_retries, order=order, config=cfg,
                                        poses=poses, out=outs, use_graph=True, arm=arm, ik=ik, gate=gate)
            call()  # capture and warm
            ctx.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            for _ in range(reps):
                call()
            e1.record(ctx.stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
        except nat.SceniError:
            continue  # shape not launchable for this batch (shared memory, occupancy)
        results.append((ms, cfg))
        if verbose:
            print(f"  {cfg}: {ms:.3f} ms", flush=True)
    return _store(cache, key, results, n)
