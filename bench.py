#!/usr/bin/env python
"""Benchmark of the Sceniris hot path on one B300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ragged|shelf|tabletop]

One step = one pass of the hot path over one batch of synthetic scene
candidates already resident in HBM. Default path (`generate`, the paper's
placement loop of Sec. IV-A with 10 retries per object, Sec. V-A): for every
object in order, sample its pose (Philox, point-in-polygon, relations), check
it against the placed objects and the world, retry the failing candidates, mark
candidates that run out of tries invalid; the first four objects of every
template must also be reachable by a 7-DoF arm (top-down grasp), decided by
exact damped-least-squares IK, with a learned gate (trained before timing on
the project's own IK labels, recall >= 0.99) skipping IK on tries it predicts
unreachable. A scene counts as verified when every object was placed by exact
collision and IK decisions. `value` is the gated, graph-replayed path;
`plain` is the same loop launched eagerly with exact IK on every try.
`kernels` times each stage's kernel alone on its own workload (exact-minimum
collision of the shelf batch, IK of 262,144 targets, gate inference and one
training epoch).

Prints ONE JSON line (rank 0). `value` is verified collision-free scenes per
second over all ranks; `e2e` is the same metric through the public C-ABI calls
with the batch copied from pinned host memory every step and the poses and
valid flags copied back (two contexts alternate, so a step's copies overlap
its neighbours' generation). `roofline` is the dominant kernel's FP32-pipe
throughput (algorithmic operations it evaluated: pair tests after the exact
sphere-level cull, sphere-box tests and the cull's own ball tests, over its
CUDA-event time) against the B300's FP32 issue peak; the stage block also
gives the throughput an exhaustive pair check would need for the same
decisions in the same time (exhaustive_equivalent_frac). `cpu_baseline` is the FP64 oracle on the host
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

# Algorithmic FP32-pipe operations per evaluated pair:
OPS_PER_SPHERE_PAIR = 5    # prune test |a|^2 - q^2 + |b|^2 - r^2 - 2a.b - 2qr: 1 FADD + 4 FFMA
OPS_PER_SPHERE_BOX = 18    # box frame (3 FADD + 3 FMUL + 6 FFMA), |p| - h (3 FADD), bound (3 FMNMX)
OPS_PER_SPHERE_BOX_COLLIDE = 15  # collision kernel: box frame (9 FFMA), |p| - h (3 FADD), bound (2 FMNMX + FSETP)
OPS_PER_POINT_TRI = 77     # point-triangle distance, face region: edges and offsets 15 FADD, six dot products 18,
                           # area terms 8, 2 divisions 8, nearest point 6 FFMA, |q|^2 3, sqrt 4, - r 1,
                           # region tests 12 FSETP, world position of the sphere 2 (FADD)
OPS_PER_CULL_TEST = 10     # sphere vs bounding ball: 3 FADD, FMUL + 2 FFMA, 2 FADD (limit), FMUL, FSETP
OPS_PER_EXHAUSTIVE_PAIR = 9  # one pair of an uncalled exhaustive check (3 FADD, FMUL + 2 FFMA, FADD, FMUL, FSETP)
OPS_PER_IK_SEED_ITER = 1000  # one check + DLS step, the scope table's algorithmic unit: FK ~315, J ~63,
                             # J J^T 147, Cholesky ~60 + 6 sqrt, solves 72, J^T y 42, error + check ~80 (FP32
                             # instructions; the 14 MUFU of the sin / cos pairs on top). The kernel's own
                             # count of the same work is ~720 (FK 280, check 40, error 21, J 63, J J^T 147,
                             # Cholesky 50, solves 60, J^T y 42, clamp 14) plus its sin / cos polynomials.
L2_BYTES = 126 * 1024 * 1024

PATHS = {
    "generate": "per-object placement loop: sample, decide collisions against placed objects and world, "
                "(designated objects) learned gate then exact IK, retry <= 10 times, invalid after that",
}

WORKLOADS = {
    "ragged": dict(make=lambda seed, T=4096: synth.ragged(seed=seed, n_templates=T), seed=2,
                   desc="ragged 4096 templates x 64 candidates, 4-64 objects, 8-128 spheres/object, convex 4-10-gon supports"),
    "shelf": dict(make=lambda seed: synth.shelf(seed=seed), seed=1,
                  desc="shelf 65536 candidates x 32 objects x 64 spheres, 25% on-top / 25% next-to, 20 world OBBs"),
    "hard": dict(make=lambda seed: synth.hard(seed=seed, n_templates=4096, n_reach=4), seed=5,
                 desc="relation-heavy 4096 templates x 64 candidates, 6-24 objects, 8-64 spheres/object, "
                      "on-top / next-to / directional / middle / face-to, convex 4-10-gon supports of 1-3 m^2"),
    "cabinet": dict(make=lambda seed: synth.cabinet(seed=seed, n_templates=4096), seed=6,
                    desc="articulated 4096 templates x 64 candidates: a counter with 4-10 objects over 2-3 drawers "
                         "(prismatic, joint values drawn every step), 2 objects inside each drawer, 16 spheres "
                         "per object, 14-19 world boxes of which 10-15 move with the drawers"),
    "meshes": dict(make=lambda seed: synth.meshes(seed=seed, n_templates=4096), seed=7,
                   desc="world-mesh 4096 templates x 64 candidates, 4-24 objects, 8-64 spheres/object, convex "
                        "4-10-gon supports of 1-3 m^2 cluttered by 2-6 box meshes (12 triangles) and 1-3 sphere "
                        "meshes (192 triangles), 216-1152 triangles per template"),
    "tabletop": dict(make=lambda seed: synth.tabletop(seed=seed), seed=0,
                     desc="tabletop 1024 candidates x 8 objects x 16 spheres on a 1.2 x 0.8 m table"),
}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate_ranks(time_s, valid, e2e_s, e2e_valid, world, device):
    """Whole-job totals over the replicas: the slowest rank's timed seconds
    (timed region and end-to-end) and the summed valid scenes."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([time_s, valid, e2e_s, e2e_valid], dtype=torch.float64, device=device)
    if world > 1:
        mx = t[[0, 2]].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t[[1, 3]].clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        t = torch.stack([mx[0], sm[0], mx[1], sm[1]])
    return [float(x) for x in t.cpu()]


def replica_seed(base_seed, rank):
    """Each rank generates an independent replica of the workload (weak scaling)."""
    return base_seed + 1000 * rank


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


# Sources each measured kernel is compiled from (a traffic record is valid
# only for the exact sources it was captured on).
KERNEL_SOURCES = {
    "reach_ik_kernel": ("generate.cu", "ik_core.cuh", "common.cuh", "kernels.h"),
    "gen_chain_kernel": ("generate.cu", "collide_core.cuh", "sample_core.cuh", "tri_core.cuh", "common.cuh",
                         "kernels.h"),
}


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2512_16896_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str):
    """DRAM bytes (read + written) per launch from profiles/traffic.json, if
    they were captured on the current sources of the kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(f"{kernel}:{workload}")
    if not d or d.get("source_hash") != kernel_source_hash(kernel):
        return None
    return d.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- oracle legs


def oracle_rate(batch, seed, budget_s: float, path: str = "generate", rng_seed: int = 0, max_retries: int = 10,
                reach: bool = False):
    """Verified collision-free scenes/s of the FP64 oracle on a bounded random
    sample of candidates (sized from a probe so the sample takes ~budget_s)."""
    import oracle
    sc = oracle.Scene(batch)
    rng = np.random.default_rng(rng_seed)
    threads = oracle.default_threads()

    def run(pick):
        if path == "generate":
            arm = oracle.make_arm(*synth.arm_arrays()) if reach else None
            ikp = oracle.ik_params(seed=seed + 3) if reach else None
            _, valid, _, _ = oracle.generate(sc, seed, max_retries=max_retries, active=pick, threads=threads, arm=arm,
                                             ikp=ikp)
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


reach_desc = ("top-down grasp of the first 4 objects of every template, 7-DoF arm at the support's -x edge, "
              "exact DLS IK (32 seeds x 100 iterations)")


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    batch = wl["make"](wl["seed"])
    reach = args.path == "generate" and not args.no_reach
    times, valids, ns, threads = [], [], [], 0
    for i in range(args.warmup + args.steps):
        r = oracle_rate(batch, seed=wl["seed"], budget_s=args.ref_step_s, path=args.path, rng_seed=100 + i,
                        max_retries=args.retries, reach=reach)
        threads = r["threads"]
        if i >= args.warmup:
            times.append(r["seconds"]); valids.append(r["valid"]); ns.append(r["n"])
    value = sum(valids) / sum(times)
    line = {
        "impl": "reference", "metric": "verified collision-free scenes/sec", "value": value, "unit": "scenes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "path": PATHS[args.path], "retries": args.retries,
                   "reachability": reach_desc if reach else None,
                   "launch": f"FP64 oracle on {threads} host threads",
                   "sample_per_step": f"{ns[0]} random candidates of the workload"},
        "cpu_baseline": {"value": value, "unit": "scenes/s", "cores": threads, "kind": "oracle",
                         "sample": f"{ns[0]} random candidates per step of the {args.workload} workload"},
        "e2e": {"value": value, "unit": "scenes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm


def in_bound_targets(seed, n, box, ikp):
    """n top-down targets drawn uniformly over box (base frame) among those the
    generation rounds' reach bounds keep: the tool within r7 + tol_pos of the
    shoulder and the wrist point t - R v within r6 + tol_pos + 2 sin(tol_rot / 2)
    |v| (r6, r7: the summed link lengths up to the wrist and the tool; v: the
    last link's offset in the tool frame), each with the rounds' 1e-5 + 1e-4."""
    d, a, alpha = (np.asarray(x, np.float64) for x in synth.arm_arrays()[:3])
    link = np.sqrt(a ** 2 + d ** 2)
    r6 = abs(a[0]) + link[1:6].sum()
    r7 = r6 + link[6]
    v = np.array([a[6], d[6] * np.sin(alpha[6]), d[6] * np.cos(alpha[6])])
    tp, tr = ikp.tol_pos + 1e-5, ikp.tol_rot + 1e-5
    b7, b6 = r7 + tp + 1e-4, r6 + tp + 2.0 * np.sin(tr / 2.0) * np.linalg.norm(v) + 1e-4
    shoulder = np.array([0.0, 0.0, d[0]])
    out, got, k = [], 0, 0
    while got < n:
        t = synth.topdown_targets(seed=seed * 1000 + k, n=max(n, 65536), box=box)
        p = t[:, 9:].astype(np.float64)
        w = p - np.einsum("nij,j->ni", t[:, :9].astype(np.float64).reshape(-1, 3, 3), v)
        keep = (np.linalg.norm(p - shoulder, axis=1) <= b7) & (np.linalg.norm(w - shoulder, axis=1) <= b6)
        out.append(t[keep])
        got += int(keep.sum())
        k += 1
    return np.ascontiguousarray(np.concatenate(out)[:n])


def run_ours(args, wl):
    import torch
    import torch.distributed as dist
    import paper_2512_16896_b300 as sc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    seed = replica_seed(wl["seed"], rank)
    batch = wl["make"](seed)
    ctx = sc.Context(local)
    stream = ctx.stream
    db = sc.DeviceBatch(batch, device=dev)
    order = torch.from_numpy(sc.order_by_work(batch)).to(dev)
    poses = db.new_poses(dev)
    n = batch.n_cand
    u8 = lambda: torch.zeros(n, dtype=torch.uint8, device=dev)
    valid, band, tries = u8(), u8(), torch.zeros(n, dtype=torch.int32, device=dev)
    q_reach = torch.zeros((db.n_poses, 7), dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    reach = args.path == "generate" and not args.no_reach
    arm = sc.make_arm(*synth.arm_arrays())
    ikp = sc.ik_params(seed=seed + 3)
    cfg = tuple(int(x) for x in args.collide_config.split(",")) if args.collide_config else None

    # ---- surrogate gate (untimed set-up: IK labels, training, threshold)
    gate = None
    gate_info = None
    rmap = None
    if reach and not args.no_gate:
        t0 = time.perf_counter()
        box = ((-0.2, 2.2), (-1.3, 1.3), (0.0, 0.8))  # base-frame region of the workload's grasp targets
        # the gate only sees tries the rounds' reach bounds keep, so it learns from those
        tr = torch.from_numpy(in_bound_targets(seed + 4, args.train_labels, box, ikp)).to(dev)
        ho = torch.from_numpy(in_bound_targets(seed + 5, 262144, box, ikp)).to(dev)
        ytr, _, _ = sc.ik_reach(ctx, arm, sc.ik_params(seed=seed + 4), tr)
        yho, _, _ = sc.ik_reach(ctx, arm, sc.ik_params(seed=seed + 5), ho)
        ctx.synchronize()
        t1 = time.perf_counter()
        gate = sc.Surrogate(ctx, seed=seed + 6)
        loss = gate.train(tr, ytr, sc.train_params(epochs=args.train_epochs, batch=4096, seed=seed + 4))
        ctx.synchronize()
        t2 = time.perf_counter()
        tau, recall, pass_rate = gate.tune_threshold(ho, yho, 0.99)
        gate_info = {"train_labels": int(tr.shape[0]), "epochs": args.train_epochs, "final_loss": float(loss[-1]),
                     "tau": tau, "heldout_recall": recall, "heldout_pass_rate": pass_rate,
                     "heldout_reachable": float(yho.float().mean().item()),
                     "targets": "top-down grasps uniform over the base-frame box, among those the rounds' reach bounds keep",
                     "label_seconds": round(t1 - t0, 2), "train_seconds": round(t2 - t1, 2),
                     "train_samples_per_s": int(args.train_epochs * tr.shape[0] / max(t2 - t1, 1e-9))}
        gate_info["vs_reach_map"], rmap = compare_gates(sc, ctx, gate, tr, ytr, ho, yho, recall, pass_rate)
        del tr, ho, ytr, yho

    # launch shape of the generation kernels: the project's autotuner times
    # whole graph-replayed calls of this workload over its search space
    # (untimed set-up) unless a shape is given
    shape_info = None
    if cfg is None and not args.no_tune:
        from paper_2512_16896_b300 import autotune
        t0 = time.perf_counter()
        cfg, tune = autotune.tune_generate(ctx, db, batch, order, seed=seed * 7919 + 7, max_retries=args.retries,
                                           arm=arm if reach else None, ik=ikp, gate=gate, verbose=args.tune_verbose)
        shape_info = {"threads": cfg[0], "a_per_lane": cfg[1], "ctas_per_sm": cfg[3], "tuned": True,
                      "tune_ms_best": round(tune["ms"], 3), "tune_seconds": round(time.perf_counter() - t0, 1),
                      "top": tune["top"][:4]}
    elif cfg is not None:
        shape_info = {"threads": cfg[0], "a_per_lane": cfg[1], "ctas_per_sm": cfg[3], "tuned": False}

    def enqueue(step_seed, use_gate=True, use_graph=True, use_map=False):
        if db.max_parts:  # a new articulation state per step, then the scenes around it
            sc.sample_parts(ctx, db, seed=step_seed)
        sc.generate(ctx, db, seed=step_seed, max_retries=args.retries, order=order, config=cfg, poses=poses,
                    out=(valid, band, tries), use_graph=use_graph and not args.no_graph,
                    arm=arm if reach else None, ik=ikp, gate=gate if use_gate and not use_map else None,
                    q_reach=q_reach if reach else None, rmap=rmap if use_map else None)

    def timed(label, use_gate, use_graph, steps, warmup, use_map=False):
        ctx.set_timing(True)
        for i in range(warmup):
            with torch.cuda.stream(stream):
                flush.zero_()
            enqueue(seed * 7919 + i, use_gate, use_graph, use_map)
        ctx.synchronize()
        if world > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        vals, stats = [], []
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # evict L2 between timed steps (not timed)
            ev[i][0].record(stream)
            enqueue(seed * 7919 + 1000 + i, use_gate, use_graph, use_map)
            ev[i][1].record(stream)
            stats.append(ctx.generate_stats())  # synchronises after the step
            tr_st, tr_a, tr_b = ctx.generate_trace()
            g_idx = np.nonzero(tr_st == 0)[0]
            # the chained launch is the step's last generation launch; the rest are the rounds
            stats[-1]["ms_chain"] = float(tr_b[g_idx[-1]] - tr_a[g_idx[-1]]) if len(g_idx) else 0.0
            vals.append(int(valid.sum().item()))
            if args.trace and i == steps - 1 and label in ("batched+surrogate", "batched"):
                st_, a_, b_ = ctx.generate_trace()
                with open(args.trace, "w") as f:
                    json.dump({"label": label, "stage": st_.tolist(), "start_ms": a_.tolist(),
                               "end_ms": b_.tolist()}, f)
        torch.cuda.synchronize()
        ctx.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        return {"label": label, "ms": ms, "valid": vals, "stats": stats}

    with ClockSampler(local) as clocks:
        main = timed("batched+surrogate" if gate is not None else "batched", gate is not None, True, args.steps,
                     args.warmup)
    plain = None
    if reach and not args.no_plain:
        plain = timed("plain", False, False, args.plain_steps, min(args.warmup, 3))
    per_tmpl = None
    if reach and not args.no_plain and args.per_template_s > 0:
        per_tmpl = plain_per_template(sc, ctx, db, batch, args, arm, ikp, seed, poses, valid, band, tries,
                                      q_reach, args.per_template_s)
    map_run = None
    if rmap is not None and args.map_steps > 0:
        map_run = timed("batched+map", False, True, args.map_steps, min(args.warmup, 3), use_map=True)
        rmap.close()

    # ---- end to end through the C ABI with host buffers. Two contexts with
    # their own device buffers alternate, so one step's copies (the batch in
    # from pinned host memory, the poses and valid flags out) overlap its
    # neighbours' generation; every step still copies its own inputs in and
    # its result out inside the timed region (inputs exceed L2, no flush).
    hb = sc.DeviceBatch(batch, pinned_host=True)
    keys = [k for k in hb.t if k != "tmpl_pose_off"]
    h2d = sum(hb.t[k].numel() * hb.t[k].element_size() for k in keys)
    d2h = poses.numel() * 4 + n
    e2e_ms, e2e_valid = [], []
    if not args.no_e2e:
        ctx.set_timing(False)
        ctxs = [ctx, sc.Context(local)]
        dbs = [db, sc.DeviceBatch(batch, device=dev)]
        outs = [(poses, valid, band, tries, q_reach),
                (dbs[1].new_poses(dev), u8(), u8(), torch.zeros(n, dtype=torch.int32, device=dev),
                 torch.zeros_like(q_reach))]
        h_poses = [torch.empty_like(poses, device="cpu").pin_memory() for _ in range(2)]
        h_valid = [torch.empty(n, dtype=torch.uint8).pin_memory() for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        total = args.warmup + args.steps
        ev_gen = [torch.cuda.Event() for _ in range(total)]
        ev_out = [torch.cuda.Event() for _ in range(total)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(total):
            j = i % 2
            if i == args.warmup:
                torch.cuda.synchronize()
                t0.record(s_in)
            if i >= 2:
                s_in.wait_event(ev_gen[i - 2])  # slot j's batch was read by step i-2
            with torch.cuda.stream(s_in):
                for k in keys:
                    dbs[j].t[k].copy_(hb.t[k], non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(s_in)
            stream.wait_event(ev_in)
            if i >= 2:
                stream.wait_event(ev_out[i - 2])  # slot j's results of step i-2 are out
            P_, V_, B_, T_, Q_ = outs[j]
            if dbs[j].max_parts:
                sc.sample_parts(ctxs[j], dbs[j], seed=seed * 7919 + 5000 + i)
            sc.generate(ctxs[j], dbs[j], seed=seed * 7919 + 5000 + i, max_retries=args.retries, order=order,
                        config=cfg, poses=P_, out=(V_, B_, T_), use_graph=not args.no_graph,
                        arm=arm if reach else None, ik=ikp, gate=gate, q_reach=Q_ if reach else None)
            ev_gen[i].record(stream)
            s_out.wait_event(ev_gen[i])
            with torch.cuda.stream(s_out):
                h_poses[j].copy_(P_, non_blocking=True)
                h_valid[j].copy_(V_, non_blocking=True)
            ev_out[i].record(s_out)
            if i >= 1:
                ev_out[i - 1].synchronize()
                if i - 1 >= args.warmup:
                    e2e_valid.append(int(h_valid[(i - 1) % 2].numpy().sum()))
        t1.record(s_out)
        t1.synchronize()
        e2e_valid.append(int(h_valid[(total - 1) % 2].numpy().sum()))
        e2e_ms.append(t0.elapsed_time(t1))
        ctxs[1].close()

    # ---- aggregate over ranks (max time, summed work)
    total_s, total_valid, e2e_s, e2e_valid_sum = aggregate_ranks(
        sum(main["ms"]) / 1000.0, sum(main["valid"]), max(sum(e2e_ms), 1e-9) / 1000.0, sum(e2e_valid), world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = read_peaks()
    sm_count = ctx.num_sms
    peak_ops = sm_count * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6  # FP32 lanes x max SM clock

    def stage_roofline(run):
        st = run["stats"]
        ms_gen = sum(s["ms_stage"][0] for s in st)
        ms_ik = sum(s["ms_stage"][2] for s in st)
        ops_gen = sum(s["sphere_pairs"] for s in st) * OPS_PER_SPHERE_PAIR + \
            sum(s["sphere_box_pairs"] for s in st) * OPS_PER_SPHERE_BOX + \
            sum(s["sphere_tri_pairs"] for s in st) * OPS_PER_POINT_TRI + \
            sum(s["cull_tests"] for s in st) * OPS_PER_CULL_TEST
        ops_exh = sum(s["exhaustive_pairs"] for s in st) * OPS_PER_EXHAUSTIVE_PAIR
        ops_ik = sum(s["ik_seed_iterations"] for s in st) * OPS_PER_IK_SEED_ITER
        rate_gen = ops_gen / max(ms_gen / 1e3, 1e-12)  # FP32-pipe operations per second
        rate_ik = ops_ik / max(ms_ik / 1e3, 1e-12)
        gen = {"kernel": "gen_round_kernel + gen_chain_kernel (sample + collision decision; the stage's work "
                         "counters cover both)", "ms_per_step": ms_gen / len(st),
               "launches_per_step": st[0]["launches_stage"][0], "achieved": rate_gen / 1e12,
               "frac": rate_gen / peak_ops,
               "exhaustive_equivalent_frac": ops_exh / max(ms_gen / 1e3, 1e-12) / peak_ops}
        ik = {"kernel": "reach_ik_kernel (DLS IK)", "ms_per_step": ms_ik / len(st),
              "launches_per_step": st[0]["launches_stage"][2], "achieved": rate_ik / 1e12, "frac": rate_ik / peak_ops}
        return gen, ik

    gen_rf, ik_rf = stage_roofline(main)
    # the dominant single kernel: the IK stage is one kernel; the generation
    # stage is two (the rounds' gen_round_kernel, the chained gen_chain_kernel)
    ms_chain = sum(s.get("ms_chain", 0.0) for s in main["stats"]) / len(main["stats"])
    gen_rf["ms_chain_per_step"] = ms_chain
    gen_rf["ms_rounds_per_step"] = gen_rf["ms_per_step"] - ms_chain
    gen_top = max(ms_chain, gen_rf["ms_per_step"] - ms_chain)
    dom = ik_rf if ik_rf["ms_per_step"] >= gen_top else gen_rf
    dom_kernel = "reach_ik_kernel" if dom is ik_rf else "gen_chain_kernel"
    clk = clocks.summary()
    cpu = None
    if world == 1 and args.cpu_budget_s > 0:
        cpu = oracle_rate(batch, seed=seed, budget_s=args.cpu_budget_s, path=args.path, max_retries=args.retries,
                          reach=reach)
    st0 = main["stats"][-1]
    plain_line = None
    if plain:
        p_s = sum(plain["ms"]) / 1000.0
        p_ik = plain["stats"][-1]
        plain_line = {"value": sum(plain["valid"]) / p_s, "unit": "scenes/s", "ms_per_step": 1000 * p_s / len(plain["ms"]),
                      "steps": len(plain["ms"]), "valid_per_step": sum(plain["valid"]) / len(plain["valid"]),
                      "ik_solves_per_step": p_ik["ik_solves"], "launch": "eager", "gate": None}
    map_line = None
    if map_run:
        m_s = sum(map_run["ms"]) / 1000.0
        m_st = map_run["stats"][-1]
        map_line = {"value": sum(map_run["valid"]) / m_s, "unit": "scenes/s",
                    "ms_per_step": 1000 * m_s / len(map_run["ms"]), "steps": len(map_run["ms"]),
                    "valid_per_step": sum(map_run["valid"]) / len(map_run["valid"]),
                    "ik_solves_per_step": m_st["ik_solves"], "gate_rejections_per_step": m_st["gate_rejections"],
                    "launch": "CUDA graph replay",
                    "gate": "4D reachability map from the same IK labels, recall >= 0.99 on the held-out targets"}
    cfg_block = {"workload": wl["desc"], "path": PATHS[args.path], "retries": args.retries,
                 "reachability": reach_desc if reach else None,
                 "gate": gate_info, "launch": "eager" if args.no_graph else "CUDA graph replay",
                 "candidates_per_gpu": n, "valid_per_step": total_valid / args.steps / world,
                 "l2": "flushed between timed steps (256 MB write, untimed); inputs exceed L2",
                 "parallelism": f"replicas x{world}",
                 "launch_shape": shape_info,
                 # the metric's own comparison as scalars: the plain paths and the gate's quality
                 "plain_value": plain_line["value"] if plain_line else None,
                 "plain_per_template_value": per_tmpl["value"] if per_tmpl else None,
                 "gate_heldout_recall": gate_info["heldout_recall"] if gate_info else None,
                 "gate_pass_rate": gate_info["heldout_pass_rate"] if gate_info else None}
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
        "config": cfg_block,
        "plain": plain_line,
        "plain_per_template": per_tmpl,
        "map_gated": map_line,
        "stages": {"gen_ms_per_step": gen_rf["ms_per_step"], "ik_ms_per_step": ik_rf["ms_per_step"],
                   "gate_ms_per_step": sum(s["ms_stage"][1] for s in main["stats"]) / len(main["stats"]),
                   "ik_solves_per_step": st0["ik_solves"], "gate_rejections_per_step": st0["gate_rejections"],
                   "reach_bound_rejections_per_step": st0["reach_bound_rejections"],
                   "sphere_pairs_per_step": st0["sphere_pairs"], "cull_tests_per_step": st0["cull_tests"],
                   "point_triangle_per_step": st0["sphere_tri_pairs"],
                   "exhaustive_pairs_per_step": st0["exhaustive_pairs"],
                   "ik_seed_iterations_per_step": st0["ik_seed_iterations"],
                   "gen_roofline_frac": gen_rf["frac"], "ik_roofline_frac": ik_rf["frac"],
                   "gen_rounds_ms_per_step": gen_rf["ms_rounds_per_step"],
                   "gen_chain_ms_per_step": gen_rf["ms_chain_per_step"],
                   "gen_exhaustive_equivalent_frac": gen_rf["exhaustive_equivalent_frac"]},
        "roofline": {"bound": "alu", "kernel": dom["kernel"], "achieved": dom["achieved"], "peak": peak_ops / 1e12,
                     "unit": "Tops/s", "frac": dom["frac"], "traffic": measured_traffic(dom_kernel, args.workload),
                     "peak_source": f"{sm_count} SMs x 128 FP32 lanes x {peaks.get('sm_max_mhz')} MHz "
                                    f"({peak_src} max clock)",
                     "ms_per_step_in_kernel": dom["ms_per_step"], "launches_per_step": dom["launches_per_step"]},
        "cpu_baseline": None if cpu is None else {
            "value": cpu["valid_per_s"], "unit": "scenes/s", "cores": cpu["threads"], "kind": "oracle",
            "sample": f"{cpu['n']} random candidates of the same workload ({cpu['seconds']:.1f} s)"},
        "e2e": None if args.no_e2e else {"value": e2e_valid_sum / e2e_s, "unit": "scenes/s",
                                          "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_step(db, args, reach, gate) * args.steps,
        "clocks": clk,
    }
    if not args.no_kernels and world == 1:
        line["kernels"] = kernel_suite(sc, ctx, dev, peak_ops)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def plain_per_template(sc, ctx, db, batch, args, arm, ikp, seed, poses, valid, band, tries, q_reach, budget_s):
    """The scope table's plain arm: the same placement loop with exact IK on
    every try, launched eagerly once per template (no batching across
    templates, no graph, no gate), over templates taken in a seeded random
    order until about budget_s seconds have run. Returns verified scenes/s
    over the candidates of the templates it ran."""
    import torch
    dev = poses.device
    rng = np.random.default_rng(seed + 77)
    order_t = rng.permutation(batch.n_templates)
    off = batch.cand_tmpl_off
    lists = [torch.arange(int(off[t]), int(off[t + 1]), dtype=torch.int32, device=dev) for t in order_t[:8]]

    def one(t_list, step_seed):
        sc.generate(ctx, db, seed=step_seed, max_retries=args.retries, order=t_list, poses=poses,
                    out=(valid, band, tries), use_graph=False, arm=arm, ik=ikp, gate=None, q_reach=q_reach)

    for i, t_list in enumerate(lists[:4]):  # warm-up
        one(t_list, seed * 7919 + 9000 + i)
    ctx.synchronize()
    valid.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(ctx.stream)
    t0 = time.perf_counter()
    done = []
    for t in order_t:
        t_list = torch.arange(int(off[t]), int(off[t + 1]), dtype=torch.int32, device=dev)
        one(t_list, seed * 7919 + 9100)
        done.append(t_list)
        if len(done) % 16 == 0:
            ctx.synchronize()
            if time.perf_counter() - t0 > budget_s:
                break
    b.record(ctx.stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    cand = torch.cat(done)
    n_valid = int(valid[cand].sum().item())
    return {"value": n_valid / (ms / 1e3), "unit": "scenes/s", "templates": len(done), "candidates": int(cand.numel()),
            "valid": n_valid, "ms": ms, "launch": "eager, one sc_generate call per template, exact IK on every try"}


def kernel_suite(sc, ctx, dev, peak_ops, only=None, shelf_cand=65536):
    """Each row's kernel alone, timed with CUDA events on the context's stream.
    only: regular expression on the row names (None: every row)."""
    import re
    import torch
    stream = ctx.stream
    out = {}
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    want = lambda key: only is None or re.search(only, key) is not None
    if any(want(f"collide_{m}_{w}") for m in ("exact_min", "decide") for w in ("shelf", "ragged", "meshes")):
        kernel_suite_collide(sc, ctx, dev, peak_ops, out, want, shelf_cand)
    if any(want(k) for k in ("ik_topdown_262144", "gate_infer_262144", "gate_train_epoch_262144",
                              "rmap_build_262144", "rmap_query_262144")):
        kernel_suite_ik_gate(sc, ctx, dev, out, want, peak_ops)
    if want("tabletop_graph_1024"):
        out["tabletop_graph_1024"] = tabletop_graph(sc, ctx, dev)
    return out


def tabletop_graph(sc, ctx, dev, replays=1000):
    """The small plain case: one tabletop template, 1024 candidates x 8
    objects x 16 spheres. One batch = sample every object's pose, then the
    whole-scene collision check (exact minimum); captured once into a CUDA
    graph and replayed `replays` times back to back: microseconds per batch
    (launch latency bound), next to the same two calls launched eagerly."""
    import torch
    stream = torch.cuda.Stream(dev)  # graphs are captured on a non-default stream
    ctx = sc.Context(dev.index if dev.index is not None else torch.cuda.current_device(), stream=stream)
    b = synth.tabletop(seed=0, n_cand=1024)
    db = sc.DeviceBatch(b, device=dev)
    poses = db.new_poses(dev)
    n = b.n_cand
    ok, sband = torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.uint8, device=dev)
    col, md, cband = (torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.float32, device=dev),
                      torch.empty(n, dtype=torch.uint8, device=dev))

    def batch_once():
        sc.sample_poses(ctx, db, seed=0, poses=poses, out=(ok, sband))
        sc.collide(ctx, db, poses, out=(col, md, cband))

    with torch.cuda.stream(stream):
        for _ in range(3):
            batch_once()
    ctx.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch_once()
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    with torch.cuda.stream(stream):
        for _ in range(10):
            g.replay()
        a, z = ev()
        a.record(stream)
        for _ in range(replays):
            g.replay()
        z.record(stream)
        z.synchronize()
        c, d = ev()
        c.record(stream)
        for _ in range(replays):
            batch_once()
        d.record(stream)
        d.synchronize()
    ctx.synchronize()
    free = int(((col == 0) & (ok == 1)).sum().item())
    ctx.close()
    us = a.elapsed_time(z) * 1e3 / replays
    return {"us_per_batch_graph": us, "us_per_batch_eager": c.elapsed_time(d) * 1e3 / replays, "replays": replays,
            "candidates": n, "collision_free": free,
            "candidates_per_s": n / (us / 1e6)}


def exhaustive_work(batch):
    """Sphere pairs between different objects and sphere-box pairs of every
    candidate of a batch (the all-pairs check the culls stand in for)."""
    so, to, bo = batch.obj_sph_off, batch.tmpl_obj_off, batch.tmpl_obb_off
    tro = batch.tmpl_tri_off if batch.tri is not None else np.zeros(len(to), np.int64)
    ncand = np.diff(batch.cand_tmpl_off)
    pairs = boxes = tris = 0
    for t in range(len(to) - 1):
        n_o = np.diff(so[to[t]:to[t + 1] + 1]).astype(np.int64)
        S = int(n_o.sum())
        pairs += int(ncand[t]) * (S * S - int((n_o * n_o).sum())) // 2
        boxes += int(ncand[t]) * S * int(bo[t + 1] - bo[t])
        tris += int(ncand[t]) * S * int(tro[t + 1] - tro[t])
    return pairs, boxes, tris


def kernel_suite_collide(sc, ctx, dev, peak_ops, out, want, shelf_cand):
    """Whole-scene collision on sampled poses, both modes: the shelf batch
    (65,536 x 32 objects x 64 spheres, 20 boxes), the ragged batch and the
    world-mesh batch."""
    import torch
    from paper_2512_16896_b300 import autotune
    stream = ctx.stream
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    for name, make in (("shelf", lambda: synth.shelf(seed=1, n_cand=shelf_cand)), ("ragged", lambda: synth.ragged(seed=2)),
                       ("meshes", lambda: synth.meshes(seed=7))):
        keys = {0: f"collide_exact_min_{name}", 1: f"collide_decide_{name}"}
        if not any(want(k) for k in keys.values()):
            continue
        batch = make()
        db = sc.DeviceBatch(batch, device=dev)
        order = torch.from_numpy(sc.order_by_work(batch)).to(dev)
        poses, _, _ = sc.sample_poses(ctx, db, seed=1)
        col = torch.empty(batch.n_cand, dtype=torch.uint8, device=dev)
        md = torch.empty(batch.n_cand, dtype=torch.float32, device=dev)
        cb = torch.empty(batch.n_cand, dtype=torch.uint8, device=dev)
        pairs_all, box_all, tri_all = exhaustive_work(batch)
        for mode, key in keys.items():
            if not want(key):
                continue
            # the project's autotuner picks the launch shape on a strided sample
            # of the LPT list (untimed); the default shape is timed beside it
            shape, tune = autotune.tune_collide(ctx, db, batch, poses, order, decide=bool(mode))
            cfg = tuple(shape)  # (threads, a_per_lane, seg_len, ctas_per_sm, decide_only, stage_bulk)

            def timed_collide(config):
                ms_, work_ = [], []
                for i in range(5):
                    with torch.cuda.stream(stream):
                        flush.zero_()
                    a, b = ev()
                    a.record(stream)
                    sc.collide(ctx, db, poses, active=order, out=(col, md, cb), config=config)
                    b.record(stream)
                    work_.append(sc.collide_last_work(ctx) + (sc.collide_last_tri_work(ctx),))
                    if i >= 2:
                        ms_.append(a.elapsed_time(b))
                return ms_, work_

            ms_def, _ = timed_collide((0, 0, 0, 0, mode))
            ms, work = timed_collide(cfg)
            t = np.mean(ms) / 1e3
            ops = np.mean([p * OPS_PER_SPHERE_PAIR + q * OPS_PER_SPHERE_BOX_COLLIDE + r * OPS_PER_POINT_TRI
                           for p, q, r in work[2:]])
            out[key] = {"ms": float(np.mean(ms)), "candidates_per_s": batch.n_cand / t,
                        "launch_shape": {"threads": shape[0], "a_per_lane": shape[1], "seg_len": shape[2],
                                         "ctas_per_sm": shape[3], "stage_bulk": shape[5], "tuned_on": tune["sample"],
                                         "top": tune["top"][:4]},
                        "ms_default_shape": float(np.mean(ms_def)),
                        "evaluated_pairs": float(np.mean([w[0] for w in work[2:]])),
                        "box_pairs": float(np.mean([w[1] for w in work[2:]])),
                        "exhaustive_pairs": float(pairs_all),
                        "exhaustive_box_pairs": float(box_all),
                        "point_triangle": float(np.mean([w[2] for w in work[2:]])),
                        "exhaustive_sphere_triangle": float(tri_all),
                        "collide_frac": float(col.float().mean().item()),
                        "roofline_frac": float(ops / t / peak_ops),
                        # every pair at the same rate: the work the bounding-ball
                        # culls save, as a fraction of the FP32 issue peak
                        "exhaustive_equivalent_frac": float((pairs_all * OPS_PER_EXHAUSTIVE_PAIR + box_all *
                                                             OPS_PER_SPHERE_BOX_COLLIDE + tri_all *
                                                             OPS_PER_POINT_TRI) / t / peak_ops)}
        del db, poses, col, md, cb


def kernel_suite_ik_gate(sc, ctx, dev, out, want, peak_ops):
    import torch
    stream = ctx.stream
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    tg = torch.from_numpy(synth.topdown_targets(seed=3, n=262144)).to(dev)
    if want("ik_topdown_262144") or want("rmap_build_262144") or want("rmap_query_262144"):
        # IK: 262,144 top-down grasp targets over the tabletop region, 32 seeds x 100 iterations
        arm = sc.make_arm(*synth.arm_arrays())
        ms = []
        for i in range(4):
            a, b = ev()
            a.record(stream)
            r, q, err = sc.ik_reach(ctx, arm, sc.ik_params(seed=3), tg)
            b.record(stream)
            b.synchronize()
            if i >= 1:
                ms.append(a.elapsed_time(b))
        seed_iters = sc.ik_last_work(ctx)
        t_ik = float(np.mean(ms)) / 1e3
        out["ik_topdown_262144"] = {"ms": float(np.mean(ms)), "targets_per_s": 262144 / t_ik,
                                    "reachable": float(r.float().mean().item()), "seed_iterations": seed_iters,
                                    "ops_per_seed_iteration": OPS_PER_IK_SEED_ITER,
                                    "roofline_frac": seed_iters * OPS_PER_IK_SEED_ITER / t_ik / peak_ops}
        # 4D reachability map from these labels: build, then query the same targets
        m = sc.ReachMap(ctx)
        bms, qms = [], []
        score = torch.empty(262144, dtype=torch.uint16, device=dev)
        for i in range(4):
            a, b = ev()
            a.record(stream)
            m.build(tg, r)
            b.record(stream)
            c, d = ev()
            c.record(stream)
            m.query(tg, out=score)
            d.record(stream)
            d.synchronize()
            if i >= 1:
                bms.append(a.elapsed_time(b))
                qms.append(c.elapsed_time(d))
        q_ms = float(np.mean(qms))
        out["rmap_build_262144"] = {"ms": float(np.mean(bms)), "labels_per_s": 262144 / (np.mean(bms) / 1e3)}
        out["rmap_query_262144"] = {"ms": q_ms, "queries_per_s": 262144 / (q_ms / 1e3),
                                    "hbm_gbs": 262144 * 58 / (q_ms / 1e3) / 1e9,
                                    "bytes_per_query": "48 in + 8 gathered + 2 out"}
        m.close()
    if not (want("gate_infer_262144") or want("gate_train_epoch_262144")):
        return
    # gate inference and one training epoch
    net = sc.Surrogate(ctx, seed=1)
    flops = 2.0 * 262144 * (9 * 256 + 2 * 256 * 256 + 256)
    if want("gate_infer_262144"):
        ms = []
        for i in range(4):
            a, b = ev()
            a.record(stream)
            net.infer(tg)
            b.record(stream)
            b.synchronize()
            if i >= 1:
                ms.append(a.elapsed_time(b))
        out["gate_infer_262144"] = {"ms": float(np.mean(ms)), "samples_per_s": 262144 / (np.mean(ms) / 1e3),
                                    "tflops": flops / (np.mean(ms) / 1e3) / 1e12}
    if want("gate_train_epoch_262144"):
        y = (torch.rand(262144, device=dev) < 0.5).to(torch.uint8)
        net.train(tg, y, sc.train_params(epochs=1, batch=4096))  # warm-up: buffers, feature moments
        torch.cuda.synchronize()
        a, b = ev()
        a.record(stream)
        net.train(tg, y, sc.train_params(epochs=1, batch=4096, seed=2))
        b.record(stream)
        b.synchronize()
        t = a.elapsed_time(b)
        out["gate_train_epoch_262144"] = {"ms": t, "samples_per_s": 262144 / (t / 1e3),
                                          "tflops": 3 * flops / (t / 1e3) / 1e12}
    net.close()


def run_kernels(args):
    """The per-kernel rows alone, on one GPU (profiling entry point)."""
    import torch
    import paper_2512_16896_b300 as sc
    torch.cuda.set_device(0)
    ctx = sc.Context(0)
    peaks, _ = read_peaks()
    peak_ops = ctx.num_sms * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6
    out = kernel_suite(sc, ctx, torch.device("cuda", 0), peak_ops, only=args.kernel_filter, shelf_cand=args.shelf_cand)
    ctx.synchronize()
    print(json.dumps({"kernels": out, "shelf_cand": args.shelf_cand}))
    ctx.close()
    return 0


def compare_gates(sc, ctx, gate, tr, ytr, ho, yho, gate_recall, gate_pass_rate):
    """The RM4D-style 4D reachability map (the paper's kind of reachability
    check, Sec. IV-E) built from the same IK labels as the learned gate, tuned
    to the same recall on the same held-out targets: recall, pass rate and
    device time per query of each, and the map's build time."""
    import torch
    stream = ctx.stream
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def timed(fn, reps=5):
        ms = []
        for i in range(reps + 1):
            a, b = ev()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if i:
                ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    m = sc.ReachMap(ctx)
    a, b = ev()
    a.record(stream)
    m.build(tr, ytr)
    b.record(stream)
    b.synchronize()
    build_ms = a.elapsed_time(b)
    tau, rec, pr = m.tune_threshold(ho, yho, 0.99)
    score = torch.empty(ho.shape[0], dtype=torch.uint16, device=ho.device)
    map_ms = timed(lambda: m.query(ho, out=score))
    gate_ms = timed(lambda: gate.infer(ho))
    out = {"queries": int(ho.shape[0]), "map_cells": m.cells, "map_build_ms": round(build_ms, 3),
           "map_tau": tau, "map_recall": rec, "map_pass_rate": pr, "map_query_ms": round(map_ms, 4),
           "gate_recall": gate_recall, "gate_pass_rate": gate_pass_rate, "gate_infer_ms": round(gate_ms, 4)}
    return out, m


def launches_per_step(db, args, reach, gate):
    """Kernels one sc_generate call enqueues: init and tables; per round of the
    objects with reachability a generation step and the reach stage (grasp
    targets, [gate forward, gate split], IK; rounds past the last candidate
    exit at once); then one chained launch for the remaining objects."""
    K, R = db.c.max_obj, args.retries
    per_round_reach = 4 if gate is not None else 2
    n_reach = min(4, K) if reach else 0
    rounds = 2 * n_reach * (R + 1)  # generate_rounds(): a try of a reach object spans two rounds
    parts = 1 if db.max_parts else 0  # sc_sample_parts before the generation call
    return parts + 2 + rounds * (1 + per_round_reach) + (1 if n_reach < K else 0)


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
    ap.add_argument("--no-tune", action="store_true",
                    help="use the library's default launch shape for generation (skip the autotuner)")
    ap.add_argument("--collide-config", type=str, default="", help="threads,a_per_lane,seg_len,ctas_per_sm")
    ap.add_argument("--tune-verbose", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the generation steps eagerly")
    ap.add_argument("--no-reach", action="store_true", help="generation without the reachability stage")
    ap.add_argument("--no-gate", action="store_true", help="no learned gate (exact IK on every try)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain (eager, ungated) comparison run")
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--map-steps", type=int, default=3, help="steps of the map-gated comparison run (0: none)")
    ap.add_argument("--no-kernels", action="store_true", help="skip the per-kernel measurements")
    ap.add_argument("--kernels-only", action="store_true",
                    help="only the per-kernel measurements (one JSON line; profiling)")
    ap.add_argument("--kernel-filter", type=str, default=None, help="regular expression on the kernel row names")
    ap.add_argument("--per-template-s", type=float, default=3.0,
                    help="seconds of the one-launch-per-template plain arm (0: skip)")
    ap.add_argument("--trace", type=str, default=None,
                    help="write the per-launch stage trace of the last timed gated step to this JSON file")
    ap.add_argument("--shelf-cand", type=int, default=65536, help="shelf candidates of the collision rows")
    ap.add_argument("--train-labels", type=int, default=4194304)
    ap.add_argument("--train-epochs", type=int, default=2)
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.workload == "ragged" and args.templates != 4096:
        T = args.templates
        wl["make"] = lambda seed: synth.ragged(seed=seed, n_templates=T)
        wl["desc"] = wl["desc"].replace("4096 templates", f"{T} templates")
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.kernels_only:
        return run_kernels(args)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
