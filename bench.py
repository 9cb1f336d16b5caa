#!/usr/bin/env python
"""Benchmark of the Sceniris hot path on one B300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ragged|shelf|tabletop] [--path generate|whole]

One step = one pass of the hot path over one batch of synthetic scene
candidates already resident in HBM. Default path (`generate`, the paper's
placement loop of Sec. IV-A with 10 retries per object, Sec. V-A): for every
object in order, sample its pose (Philox, point-in-polygon, relations), check
it against the placed objects and the world, retry the failing candidates, mark
candidates that run out of tries invalid. A scene counts as verified
collision-free when every object was placed by exact decisions. `--path whole`
times the plain whole-scene pass instead (sample every object, then the exact
minimum distance of every candidate).

Prints ONE JSON line (rank 0). `value` is verified collision-free scenes per
second over all ranks; `e2e` is the same metric through the public C-ABI calls
with the batch copied from pinned host memory every step and the poses and
valid flags copied back. `roofline` is the dominant kernel's FP32-pipe
throughput (algorithmic operations it evaluated / its CUDA-event time) against
the B300's FP32 issue peak. `cpu_baseline` is the FP64 oracle on the host
cores over a bounded random sample of the same workload.

--impl reference runs that oracle (as it is) as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# Algorithmic FP32-pipe operations per evaluated pair ("Rooflines"):
OPS_PER_SPHERE_PAIR = 5    # prune test |a|^2 - q^2 + |b|^2 - r^2 - 2a.b - 2qr: 1 FADD + 4 FFMA
OPS_PER_SPHERE_BOX = 18    # box frame (3 FADD + 3 FMUL + 6 FFMA), |p| - h (3 FADD), bound (3 FMNMX)
L2_BYTES = 126 * 1024 * 1024

PATHS = {
    "generate": "per-object placement loop: sample, decide collisions against placed objects and world, "
                "retry <= 10 times, invalid after that",
    "whole": "plain whole-scene: sample all objects, one exact-minimum collision pass",
}

WORKLOADS = {
    "ragged": dict(make=lambda seed, T=4096: synth.ragged(seed=seed, n_templates=T), seed=2,
                   desc="ragged 4096 templates x 64 candidates, 4-64 objects, 8-128 spheres/object, convex 4-10-gon supports"),
    "shelf": dict(make=lambda seed: synth.shelf(seed=seed), seed=1,
                  desc="shelf 65536 candidates x 32 objects x 64 spheres, 25% on-top / 25% next-to, 20 world OBBs"),
    "tabletop": dict(make=lambda seed: synth.tabletop(seed=seed), seed=0,
                     desc="tabletop 1024 candidates x 8 objects x 16 spheres on a 1.2 x 0.8 m table"),
}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active"
    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
               0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
                bits = int(parts[3], 16)
            except ValueError:
                continue
            for b, n in self.REASONS.items():
                if bits & b and n != "gpu_idle":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash(name: str) -> str:
    p = os.path.join(ROOT, "paper_2512_16896_b300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def measured_traffic(kernel_file: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of the kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(f"{kernel_file}:{workload}")
    if not d or d.get("source_hash") != kernel_source_hash(kernel_file):
        return None
    return d.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- oracle legs


def oracle_rate(batch, seed, budget_s: float, path: str = "generate", rng_seed: int = 0, max_retries: int = 10):
    """Verified collision-free scenes/s of the FP64 oracle on a bounded random
    sample of candidates (sized from a probe so the sample takes ~budget_s)."""
    import oracle
    sc = oracle.Scene(batch)
    rng = np.random.default_rng(rng_seed)
    threads = oracle.default_threads()

    def run(pick):
        if path == "generate":
            _, valid, _, _ = oracle.generate(sc, seed, max_retries=max_retries, active=pick, threads=threads)
            return int(valid.sum())
        P, ok, _ = oracle.sample_poses(sc, seed, active=pick, threads=threads)
        col, md, _ = oracle.collide(sc, P, active=pick, threads=threads)
        return int(np.sum(ok.astype(bool) & (md >= 0)))

    probe = rng.choice(batch.n_cand, min(batch.n_cand, 4 * threads), replace=False).astype(np.int32)
    run(probe[: 2 * threads])  # load and warm the library
    t0 = time.perf_counter()
    run(probe)
    dt = max(time.perf_counter() - t0, 1e-3)
    n = int(min(batch.n_cand, max(len(probe), len(probe) * budget_s / dt)))
    pick = rng.choice(batch.n_cand, n, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    valid = run(pick)
    dt = time.perf_counter() - t0
    return {"valid": valid, "n": n, "seconds": dt, "threads": threads,
            "scenes_per_s": n / dt, "valid_per_s": valid / dt}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    batch = wl["make"](wl["seed"])
    times, valids, ns = [], [], []
    for i in range(args.warmup + args.steps):
        r = oracle_rate(batch, seed=wl["seed"], budget_s=args.ref_step_s, path=args.path, rng_seed=100 + i,
                        max_retries=args.retries)
        if i >= args.warmup:
            times.append(r["seconds"]); valids.append(r["valid"]); ns.append(r["n"])
    value = sum(valids) / sum(times)
    line = {
        "impl": "reference", "metric": "verified collision-free scenes/sec", "value": value, "unit": "scenes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "path": PATHS[args.path], "retries": args.retries,
                   "launch": ("eager" if args.no_graph else "CUDA graph replay") if gen else "eager",
                   "sample_per_step": f"{ns[0]} random candidates of the workload"},
        "cpu_baseline": {"value": value, "unit": "scenes/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{ns[0]} random candidates per step of the {args.workload} workload"},
        "e2e": {"value": value, "unit": "scenes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm


def run_ours(args, wl):
    import torch
    import torch.distributed as dist
    import paper_2512_16896_b300 as sc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    seed = wl["seed"] + 1000 * rank  # independent replica per rank (weak scaling)
    batch = wl["make"](seed)
    ctx = sc.Context(local)
    stream = ctx.stream
    db = sc.DeviceBatch(batch, device=dev)
    order = torch.from_numpy(sc.order_by_work(batch)).to(dev)
    poses = db.new_poses(dev)
    n = batch.n_cand
    u8 = lambda: torch.zeros(n, dtype=torch.uint8, device=dev)
    valid, band, tries = u8(), u8(), torch.zeros(n, dtype=torch.int32, device=dev)
    ok, sband, col, cband = u8(), u8(), u8(), u8()
    md = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    gen = args.path == "generate"

    # launch shape: explicit, autotuned on a sample of this batch, or the default
    cfg = None
    tune_info = "library default"
    if args.collide_config:
        cfg = tuple(int(x) for x in args.collide_config.split(","))
        tune_info = "given"
    elif not args.no_tune and not gen:
        from paper_2512_16896_b300 import autotune
        sc.sample_poses(ctx, db, seed=seed, poses=poses)
        cfg, entry = autotune.tune_collide(ctx, db, batch, poses, order, verbose=args.tune_verbose)
        tune_info = f"autotuned ({entry['sample']} sampled candidates, {entry['ms']:.2f} ms)"

    def enqueue(step_seed, ev=None):
        """One step on the device; ev = (start, end) events around the dominant kernel(s)."""
        if gen:
            if ev:
                ev[0].record(stream)
            sc.generate(ctx, db, seed=step_seed, max_retries=args.retries, order=order, config=cfg, poses=poses,
                        out=(valid, band, tries), use_graph=not args.no_graph)
            if ev:
                ev[1].record(stream)
        else:
            sc.sample_poses(ctx, db, seed=step_seed, poses=poses, out=(ok, sband))
            if ev:
                ev[0].record(stream)
            sc.collide(ctx, db, poses, active=order, out=(col, md, cband), config=cfg)
            if ev:
                ev[1].record(stream)

    ok_by_list = torch.empty(n, dtype=torch.uint8, device=dev)

    def count_valid():
        if gen:
            return int(valid.sum().item())
        torch.index_select(ok, 0, order.long(), out=ok_by_list)  # collide outputs are in list order
        return int(((ok_by_list == 1) & (col == 0)).sum().item())

    for i in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        enqueue(seed * 7919 + i)
    torch.cuda.synchronize()
    ctx.synchronize()
    if world > 1:
        dist.barrier()

    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev_kern = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    valids, pairs, boxes = [], [], []
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # evict L2 between timed steps (not timed)
            ev_step[i][0].record(stream)
            enqueue(seed * 7919 + 1000 + i, ev_kern[i])
            ev_step[i][1].record(stream)
            p, bx = sc.collide_last_work(ctx)  # synchronises after the step's end event
            pairs.append(p)
            boxes.append(bx)
            valids.append(count_valid())
        torch.cuda.synchronize()
    ctx.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    kern_ms = [a.elapsed_time(b) for a, b in ev_kern]
    total_s = sum(step_ms) / 1000.0
    total_valid = sum(valids)

    # ---- end to end through the C ABI with host buffers
    hb = sc.DeviceBatch(batch, pinned_host=True)
    h2d = sum(t.numel() * t.element_size() for k, t in hb.t.items() if k != "tmpl_pose_off")
    h_poses = torch.empty_like(poses, device="cpu").pin_memory()
    h_valid = torch.empty(n, dtype=torch.uint8).pin_memory()
    d2h = h_poses.numel() * 4 + n
    e2e_ms, e2e_valid = [], []
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
        e0.record(stream)
        with torch.cuda.stream(stream):
            for k, t in hb.t.items():
                if k != "tmpl_pose_off":
                    db.t[k].copy_(t, non_blocking=True)
        enqueue(seed * 7919 + 5000 + i)
        with torch.cuda.stream(stream):
            h_poses.copy_(poses, non_blocking=True)
            if gen:
                h_valid.copy_(valid, non_blocking=True)
            else:
                torch.index_select(ok, 0, order.long(), out=ok_by_list)
                h_valid.copy_((ok_by_list == 1) & (col == 0), non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
            e2e_valid.append(int(h_valid.numpy().sum()))

    # ---- aggregate over ranks (max time, summed work)
    stats = torch.tensor([total_s, total_valid, max(sum(e2e_ms), 1e-9) / 1000.0, sum(e2e_valid)], dtype=torch.float64,
                         device=dev)
    if world > 1:
        mx = stats[[0, 2]].clone(); dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = stats[[1, 3]].clone(); dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        stats = torch.stack([mx[0], sm[0], mx[1], sm[1]])
    total_s, total_valid, e2e_s, e2e_valid_sum = [float(x) for x in stats.cpu()]
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = read_peaks()
    sm_count = ctx.num_sms
    peak_ops = sm_count * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6  # FP32 lanes x max SM clock
    ops = np.array(pairs, np.float64) * OPS_PER_SPHERE_PAIR + np.array(boxes, np.float64) * OPS_PER_SPHERE_BOX
    achieved = float(np.sum(ops) / (np.sum(kern_ms) / 1000.0))
    clk = clocks.summary()
    cpu = None
    if world == 1 and args.cpu_budget_s > 0:
        cpu = oracle_rate(batch, seed=seed, budget_s=args.cpu_budget_s, path=args.path, max_retries=args.retries)
    kname = "gen_step_kernel (+ its sampling)" if gen else "collide_kernel"
    launches_per_step = (1 + db.c.max_obj * (args.retries + 1)) if gen else 2
    line = {
        "metric": "verified collision-free scenes/sec",
        "value": total_valid / total_s,
        "unit": "scenes/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000 * total_s / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "path": PATHS[args.path], "retries": args.retries,
                   "launch": ("eager" if args.no_graph else "CUDA graph replay") if gen else "eager",
                   "collide_launch": {"shape": list(cfg) if cfg else None, "source": tune_info},
                   "candidates_per_gpu": n, "valid_per_step": total_valid / args.steps / world,
                   "l2": "flushed between timed steps (256 MB write, untimed); inputs exceed L2",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s", "frac": achieved / peak_ops,
                     "traffic": measured_traffic("generate.cu" if gen else "collide.cu", args.workload),
                     "peak_source": f"{sm_count} SMs x 128 FP32 lanes x {peaks.get('sm_max_mhz')} MHz "
                                    f"({peak_src} max clock)",
                     "ms_per_step_in_kernel": float(np.mean(kern_ms)),
                     "pairs_per_step": float(np.mean(pairs)), "box_pairs_per_step": float(np.mean(boxes))},
        "cpu_baseline": None if cpu is None else {
            "value": cpu["valid_per_s"], "unit": "scenes/s", "cores": cpu["threads"], "kind": "oracle",
            "sample": f"{cpu['n']} random candidates of the same workload ({cpu['seconds']:.1f} s)"},
        "e2e": None if args.no_e2e else {"value": e2e_valid_sum / e2e_s, "unit": "scenes/s",
                                          "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ragged")
    ap.add_argument("--path", choices=sorted(PATHS), default="generate")
    ap.add_argument("--retries", type=int, default=10)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--templates", type=int, default=4096, help="ragged workload: number of templates (profiling)")
    ap.add_argument("--no-tune", action="store_true", help="use the library's default collide launch shape")
    ap.add_argument("--collide-config", type=str, default="", help="threads,a_per_lane,seg_len,ctas_per_sm")
    ap.add_argument("--tune-verbose", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the generation steps eagerly")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.workload == "ragged" and args.templates != 4096:
        T = args.templates
        wl["make"] = lambda seed: synth.ragged(seed=seed, n_templates=T)
        wl["desc"] = wl["desc"].replace("4096 templates", f"{T} templates")
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
