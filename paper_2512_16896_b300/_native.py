"""ctypes view of include/sceniris.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsceniris_b300.so")

SC_OK, SC_ERR_INVALID, SC_ERR_OOM, SC_ERR_CUDA, SC_ERR_TIMEOUT, SC_ERR_UNSUPPORTED, SC_ERR_DEVICE = range(7)
_NAMES = ["SC_OK", "SC_ERR_INVALID", "SC_ERR_OOM", "SC_ERR_CUDA", "SC_ERR_TIMEOUT", "SC_ERR_UNSUPPORTED",
          "SC_ERR_DEVICE"]

_lock = threading.Lock()
_lib = None


class SceniError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES[status] if 0 <= status < len(_NAMES) else status}: {msg}")
        self.status = status


P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64


class ScSceneBatch(ctypes.Structure):
    _fields_ = [(n, I32) for n in ("n_templates", "n_objects", "n_spheres", "n_verts", "n_obb", "n_cand", "max_obj",
                                   "max_sph")] + [
        (n, P) for n in ("tmpl_obj_off", "obj_sph_off", "sph_local", "obj_half", "obj_rel", "obj_rel_param",
                         "tmpl_poly_off", "poly_verts", "tmpl_support_z", "tmpl_obb_off", "obb", "cand_tmpl_off",
                         "tmpl_pose_off", "tmpl_base", "obj_rel_dir", "obj_anchor_off", "obj_anchor")] + [
        ("n_parts", I32), ("max_parts", I32)] + [(n, P) for n in ("tmpl_part_off", "part_param", "obb_part", "part_q")] + [
        ("n_tri", I32), ("tmpl_tri_off", P), ("tri", P)]


class ScSampleParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("max_attempts", I32), ("retry", I32), ("first_obj", I32), ("n_obj", I32)]


class ScGenStats(ctypes.Structure):
    _fields_ = [("sphere_pairs", I64), ("sphere_box_pairs", I64), ("ik_solves", I64), ("gate_rejections", I64),
                ("ik_seed_iterations", I64), ("ms_stage", ctypes.c_float * 3), ("launches_stage", I32 * 3),
                ("cull_tests", I64), ("exhaustive_pairs", I64), ("sphere_tri_pairs", I64),
                ("reach_bound_rejections", I64)]

    def as_dict(self):
        return {"sphere_pairs": self.sphere_pairs, "sphere_box_pairs": self.sphere_box_pairs,
                "ik_solves": self.ik_solves, "gate_rejections": self.gate_rejections,
                "ik_seed_iterations": self.ik_seed_iterations, "ms_stage": list(self.ms_stage),
                "launches_stage": list(self.launches_stage), "cull_tests": self.cull_tests,
                "exhaustive_pairs": self.exhaustive_pairs, "sphere_tri_pairs": self.sphere_tri_pairs,
                "reach_bound_rejections": self.reach_bound_rejections}


class ScRmapParams(ctypes.Structure):
    _fields_ = [("nz", I32), ("nc", I32), ("nxy", I32), ("z_lo", ctypes.c_float), ("z_hi", ctypes.c_float),
                ("r_max", ctypes.c_float)]


class ScGenReach(ctypes.Structure):
    _fields_ = [("arm", P), ("ik", P), ("gate", P), ("map", P)]


class ScGenParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("max_attempts", I32), ("max_retries", I32), ("use_graph", I32)]


class ScArm(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float * 7) for n in ("dh_d", "dh_a", "dh_alpha", "qmin", "qmax")]


class ScIkParams(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_float), ("tol_pos", ctypes.c_float), ("tol_rot", ctypes.c_float), ("iters", I32),
                ("seeds", I32), ("seed", ctypes.c_uint64)]


def make_arm(d, a, alpha, qmin, qmax) -> ScArm:
    f = lambda v: (ctypes.c_float * 7)(*[float(x) for x in v])
    return ScArm(f(d), f(a), f(alpha), f(qmin), f(qmax))


def ik_params(lam=0.05, tol_pos=5e-3, tol_rot=0.05, iters=100, seeds=32, seed=3) -> ScIkParams:
    return ScIkParams(lam, tol_pos, tol_rot, iters, seeds, seed)


class ScTrainParams(ctypes.Structure):
    _fields_ = [("epochs", I32), ("batch", I32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("seed", ctypes.c_uint64)]


def train_params(epochs=4, batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=4) -> ScTrainParams:
    return ScTrainParams(epochs, batch, lr, beta1, beta2, eps, seed)


class CollideConfig(ctypes.Structure):
    _fields_ = [("threads", I32), ("a_per_lane", I32), ("seg_len", I32), ("ctas_per_sm", I32), ("decide_only", I32),
                ("stage_bulk", I32)]

    def as_tuple(self):
        return (self.threads, self.a_per_lane, self.seg_len, self.ctas_per_sm, self.decide_only, self.stage_bulk)


# name -> (restype, argtypes); mirrors include/sceniris.h
SIGNATURES = {
    "sc_version": (I32, []),
    "sc_last_error": (ctypes.c_char_p, []),
    "sc_ctx_create": (ctypes.c_int, [ctypes.c_int, P, ctypes.POINTER(P)]),
    "sc_ctx_destroy": (None, [P]),
    "sc_ctx_set_stream": (ctypes.c_int, [P, P]),
    "sc_ctx_synchronize": (ctypes.c_int, [P]),
    "sc_ctx_num_sms": (I32, [P]),
    "sc_sample_poses": (ctypes.c_int, [P, ctypes.POINTER(ScSceneBatch), ctypes.POINTER(ScSampleParams), P, I32, P, P,
                                       P]),
    "sc_collide": (ctypes.c_int, [P, ctypes.POINTER(ScSceneBatch), P, P, I32, I32, P, P, P]),
    "sc_collide_ex": (ctypes.c_int, [P, ctypes.POINTER(ScSceneBatch), P, P, I32, I32, ctypes.POINTER(CollideConfig), P,
                                     P, P]),
    "sc_collide_last_work": (ctypes.c_int, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "sc_collide_last_tri_work": (ctypes.c_int, [P, ctypes.POINTER(I64)]),
    "sc_order_by_work": (ctypes.c_int, [I32, P, P, P, P]),
    "sc_generate": (ctypes.c_int, [P, ctypes.POINTER(ScSceneBatch), ctypes.POINTER(ScGenParams), P, I32,
                                   ctypes.POINTER(CollideConfig), ctypes.POINTER(ScGenReach), P, P, P, P, P]),
    "sc_ik_reach": (ctypes.c_int, [P, ctypes.POINTER(ScArm), ctypes.POINTER(ScIkParams), P, P, I32, P, P, P, P]),
    "sc_ik_dls_step": (ctypes.c_int, [P, ctypes.POINTER(ScArm), ctypes.c_float, P, P, I32, P, P]),
    "sc_ik_last_work": (ctypes.c_int, [P, ctypes.POINTER(I64)]),
    "sc_mlp_param_count": (I32, []),
    "sc_mlp_create": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(P)]),
    "sc_mlp_destroy": (None, [P]),
    "sc_mlp_get": (ctypes.c_int, [P, P, P, P, P, P]),
    "sc_mlp_set": (ctypes.c_int, [P, P, P, P, P, ctypes.c_float]),
    "sc_surrogate_infer": (ctypes.c_int, [P, P, P, I32, P]),
    "sc_surrogate_grads": (ctypes.c_int, [P, P, P, P, I32, P, P]),
    "sc_mlp_adam_step": (ctypes.c_int, [P, P, P, ctypes.POINTER(ScTrainParams)]),
    "sc_mlp_train_step": (ctypes.c_int, [P, P, P, P, I32, ctypes.POINTER(ScTrainParams), P]),
    "sc_surrogate_train": (ctypes.c_int, [P, P, P, P, I32, ctypes.POINTER(ScTrainParams), P]),
    "sc_surrogate_tune_threshold": (ctypes.c_int, [P, P, P, P, I32, ctypes.c_float, P, P, P]),
    "sc_mlp_save": (ctypes.c_int, [P, P, ctypes.c_char_p]),
    "sc_mlp_load": (ctypes.c_int, [P, ctypes.c_char_p, ctypes.POINTER(P)]),
    "sc_generate_stats": (ctypes.c_int, [P, ctypes.POINTER(ScGenStats)]),
    "sc_ctx_set_timing": (ctypes.c_int, [P, I32]),
    "sc_generate_trace": (ctypes.c_int, [P, I32, ctypes.POINTER(I32), P, P, P]),
    "sc_collide_noalloc": (ctypes.c_int, [P, ctypes.POINTER(ScSceneBatch), P, P, I32, I32, P, P, P]),
    "sc_sample_parts": (ctypes.c_int, [P, ctypes.POINTER(ScSceneBatch), ctypes.c_uint64, P, I32, P]),
    "sc_rmap_create": (ctypes.c_int, [P, ctypes.POINTER(ScRmapParams), ctypes.POINTER(P)]),
    "sc_rmap_destroy": (None, [P]),
    "sc_rmap_cells": (I64, [P]),
    "sc_rmap_build": (ctypes.c_int, [P, P, P, P, I32]),
    "sc_rmap_query": (ctypes.c_int, [P, P, P, I32, P]),
    "sc_rmap_tune_threshold": (ctypes.c_int, [P, P, P, P, I32, ctypes.c_float, P, P, P]),
    "sc_rmap_get_counts": (ctypes.c_int, [P, P, P]),
    "sc_rmap_set_threshold": (ctypes.c_int, [P, I32]),
}


def lib():
    """The loaded library (raises if it is not built; there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is not built; run python -m paper_2512_16896_b300.build")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != SC_OK:
        raise SceniError(status, lib().sc_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


class Context:
    """An sc_ctx on one device, enqueuing on torch's current stream for that device."""

    def __init__(self, device: int | None = None, stream: torch.cuda.Stream | None = None):
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream or torch.cuda.current_stream(self.device)
        h = P()
        _check(lib().sc_ctx_create(self.device, P(self.stream.cuda_stream), ctypes.byref(h)))
        self.handle = h

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        _check(lib().sc_ctx_set_stream(self.handle, P(stream.cuda_stream)))

    def synchronize(self):
        _check(lib().sc_ctx_synchronize(self.handle))

    def set_timing(self, on: bool):
        _check(lib().sc_ctx_set_timing(self.handle, int(on)))

    def generate_stats(self) -> dict:
        st = ScGenStats()
        _check(lib().sc_generate_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def generate_trace(self, cap: int = 8192):
        """Per-launch trace of the last timed generate call: (stage, start_ms, end_ms) numpy arrays."""
        import numpy as np
        n = I32()
        stage = np.zeros(cap, np.int32)
        t0 = np.zeros(cap, np.float32)
        t1 = np.zeros(cap, np.float32)
        _check(lib().sc_generate_trace(self.handle, cap, ctypes.byref(n), stage.ctypes.data, t0.ctypes.data,
                                       t1.ctypes.data))
        m = min(n.value, cap)
        return stage[:m], t0[:m], t1[:m]

    @property
    def num_sms(self) -> int:
        return lib().sc_ctx_num_sms(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().sc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceBatch:
    """Device copies of a scene batch's CSR arrays (any object with the fields
    of sc_scene_batch as numpy arrays) and the sc_scene_batch that points at them."""

    FIELDS = {"tmpl_obj_off": torch.int32, "obj_sph_off": torch.int32, "sph_local": torch.float32,
              "obj_half": torch.float32, "obj_rel": torch.int32, "obj_rel_param": torch.float32,
              "tmpl_poly_off": torch.int32, "poly_verts": torch.float32, "tmpl_support_z": torch.float32,
              "tmpl_obb_off": torch.int32, "obb": torch.float32, "cand_tmpl_off": torch.int32,
              "tmpl_base": torch.float32}
    OPTIONAL = {"obj_rel_dir": torch.float32, "obj_anchor_off": torch.int32, "obj_anchor": torch.int32,
                "tmpl_part_off": torch.int32, "part_param": torch.float32, "obb_part": torch.int32,
                "tmpl_tri_off": torch.int32, "tri": torch.float32}

    def __init__(self, batch, device: int | str | torch.device = "cuda", pinned_host: bool = False):
        self.t = {}
        for name, dt in self.FIELDS.items():
            a = np.ascontiguousarray(getattr(batch, name))
            x = torch.from_numpy(a).to(dt)
            if x.numel() == 0:
                x = torch.zeros(16, dtype=dt)  # keep a valid aligned pointer for empty arrays
            self.t[name] = x.to(device) if not pinned_host else x.pin_memory()
        for name, dt in self.OPTIONAL.items():  # relation arrays a batch may leave out (NULL)
            a = getattr(batch, name, None)
            if a is not None and np.asarray(a).size:
                self.t[name] = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
                self.t[name] = self.t[name].to(device) if not pinned_host else self.t[name].pin_memory()
        if "obj_anchor" not in self.t:  # no MIDDLE object: neither anchor array
            self.t.pop("obj_anchor_off", None)
        # CSR consistency of the optional arrays (the library reads them on the
        # device, where it cannot check their lengths)
        n_t_ = len(batch.tmpl_obj_off) - 1
        tro, tri = getattr(batch, "tmpl_tri_off", None), getattr(batch, "tri", None)
        if tri is not None and np.asarray(tri).size and (
                tro is None or len(tro) != n_t_ + 1 or int(tro[-1]) != np.asarray(tri).reshape(-1, 12).shape[0]):
            raise ValueError("tmpl_tri_off must have n_templates + 1 entries ending at the triangle count")
        po, pp = getattr(batch, "tmpl_part_off", None), getattr(batch, "part_param", None)
        if pp is not None and np.asarray(pp).size:
            if po is None or len(po) != n_t_ + 1 or int(po[-1]) != np.asarray(pp).reshape(-1, 12).shape[0]:
                raise ValueError("tmpl_part_off must have n_templates + 1 entries ending at the part count")
            ob = getattr(batch, "obb_part", None)
            if ob is not None and np.asarray(ob).size and len(ob) != len(batch.obb):
                raise ValueError("obb_part needs one entry per world box")
        # articulated parts: their per-candidate joint values live next to the batch
        part_off = getattr(batch, "tmpl_part_off", None)
        n_parts_t = np.diff(part_off) if part_off is not None and len(part_off) > 1 else np.zeros(1, np.int64)
        self.max_parts = int(n_parts_t.max()) if "part_param" in self.t else 0
        if self.max_parts > 0:  # the batch's joint values, or zeros for sample_parts to fill
            q0 = getattr(batch, "part_q", None)
            n_q = int(batch.cand_tmpl_off[-1]) * self.max_parts
            q = (torch.from_numpy(np.ascontiguousarray(q0, np.float32)).reshape(-1) if q0 is not None else
                 torch.zeros(n_q, dtype=torch.float32))
            if q.numel() != n_q:  # the library reads part_q[c * max_parts + j] for every candidate
                raise ValueError(f"part_q has {q.numel()} values, the batch needs n_cand x max_parts = {n_q}")
            self.t["part_q"] = q.to(device) if not pinned_host else q.pin_memory()
        else:
            for name in ("tmpl_part_off", "part_param", "obb_part"):
                self.t.pop(name, None)
        tpo = np.concatenate([[0], np.cumsum(np.diff(batch.cand_tmpl_off).astype(np.int64) *
                                             np.diff(batch.tmpl_obj_off).astype(np.int64))]).astype(np.int64)
        self.t["tmpl_pose_off"] = torch.from_numpy(tpo).to(device)
        self.tmpl_obj_off = np.asarray(batch.tmpl_obj_off, np.int32)
        self.obj_sph_off = np.asarray(batch.obj_sph_off, np.int32)
        self.cand_tmpl_off = np.asarray(batch.cand_tmpl_off, np.int32)
        n_t = len(self.tmpl_obj_off) - 1
        nobj = np.diff(self.tmpl_obj_off)
        nsph = self.obj_sph_off[self.tmpl_obj_off[1:]] - self.obj_sph_off[self.tmpl_obj_off[:-1]]
        self.n_poses = int(tpo[-1])
        self.n_cand = int(self.cand_tmpl_off[-1])
        if "tri" not in self.t:  # no world meshes: neither triangle array
            self.t.pop("tmpl_tri_off", None)
        ptrs = {n: _ptr(self.t.get(n)) for n, _ in ScSceneBatch._fields_[8:]
                if n not in ("n_parts", "max_parts", "n_tri")}
        self.c = ScSceneBatch(
            n_t, len(batch.obj_half), len(batch.sph_local), len(batch.poly_verts), len(batch.obb), self.n_cand,
            int(nobj.max()), int(nsph.max()))
        for n, v in ptrs.items():
            setattr(self.c, n, v)
        self.c.n_parts = len(batch.part_param) if self.max_parts else 0
        self.c.max_parts = self.max_parts
        self.c.n_tri = self.t["tri"].numel() // 12 if "tri" in self.t else 0
        if len(batch.obb) == 0:
            self.c.obb = None

    @property
    def part_q(self) -> torch.Tensor | None:
        """Joint values of the articulated parts, float [n_cand][max_parts] (None without parts)."""
        q = self.t.get("part_q")
        return None if q is None else q.view(self.n_cand, self.max_parts)

    def new_poses(self, device="cuda") -> torch.Tensor:
        return torch.zeros((self.n_poses, 4), dtype=torch.float32, device=device)


def _n_items(db: DeviceBatch, active):
    return db.n_cand if active is None else int(active.numel())


_EMPTY = {}


def _active_ptr(active):
    """Device pointer of an active list; an empty list gets a valid placeholder
    pointer (NULL would mean "all candidates")."""
    if active is None:
        return None
    if active.numel() == 0:
        dev = active.device
        if dev not in _EMPTY:
            _EMPTY[dev] = torch.zeros(4, dtype=torch.int32, device=dev)
        return _ptr(_EMPTY[dev])
    assert active.dtype == torch.int32 and active.is_contiguous()
    return _ptr(active)


def sample_poses(ctx: Context, db: DeviceBatch, seed: int, max_attempts: int = 16, retry: int = 0, first_obj: int = 0,
                 n_obj: int = 1 << 30, active: torch.Tensor | None = None, poses: torch.Tensor | None = None,
                 out=None):
    """sc_sample_poses. Returns (poses [P,4] f32, sample_ok [n] u8, band [n] u8) on the device."""
    dev = torch.device("cuda", ctx.device)
    poses = db.new_poses(dev) if poses is None else poses
    n = _n_items(db, active)
    if out is None:
        ok = torch.empty(n, dtype=torch.uint8, device=dev)
        band = torch.empty(n, dtype=torch.uint8, device=dev)
    else:
        ok, band = out
    p = ScSampleParams(seed, max_attempts, retry, first_obj, n_obj)
    _check(lib().sc_sample_poses(ctx.handle, ctypes.byref(db.c), ctypes.byref(p), _active_ptr(active), n, _ptr(poses),
                                 _ptr(ok), _ptr(band)))
    return poses, ok, band


def collide(ctx: Context, db: DeviceBatch, poses: torch.Tensor, active: torch.Tensor | None = None, first_new: int = 0,
            config: CollideConfig | tuple | None = None, out=None):
    """sc_collide_ex. Returns (collide [n] u8, min_dist [n] f32, band [n] u8) on the device."""
    dev = torch.device("cuda", ctx.device)
    n = _n_items(db, active)
    if out is None:
        col = torch.empty(n, dtype=torch.uint8, device=dev)
        md = torch.empty(n, dtype=torch.float32, device=dev)
        band = torch.empty(n, dtype=torch.uint8, device=dev)
    else:
        col, md, band = out
    cfg = None
    if config is not None:
        cfg = config if isinstance(config, CollideConfig) else CollideConfig(*config)
    _check(lib().sc_collide_ex(ctx.handle, ctypes.byref(db.c), _ptr(poses), _active_ptr(active), n, first_new,
                               None if cfg is None else ctypes.byref(cfg), _ptr(col), _ptr(md), _ptr(band)))
    return col, md, band


def generate(ctx: Context, db: DeviceBatch, seed: int, max_attempts: int = 16, max_retries: int = 10,
             order: torch.Tensor | None = None, config=None, poses: torch.Tensor | None = None, out=None,
             use_graph: bool = True, arm=None, ik=None, gate=None, q_reach: torch.Tensor | None = None,
             rmap=None):
    """sc_generate. Returns (poses [P,4] f32, valid [n_cand] u8, band [n_cand] u8, tries [n_cand] i32).
    With `arm` (and `ik`), designated objects must also be reachable; `gate` (a
    Surrogate) or `rmap` (a ReachMap) filters tries before IK; q_reach [P,7]
    receives the IK solutions."""
    dev = torch.device("cuda", ctx.device)
    poses = db.new_poses(dev) if poses is None else poses
    if out is None:
        valid = torch.zeros(db.n_cand, dtype=torch.uint8, device=dev)
        band = torch.zeros(db.n_cand, dtype=torch.uint8, device=dev)
        tries = torch.zeros(db.n_cand, dtype=torch.int32, device=dev)
    else:
        valid, band, tries = out
    cfg = None
    if config is not None:
        cfg = config if isinstance(config, CollideConfig) else CollideConfig(*config)
    p = ScGenParams(seed, max_attempts, max_retries, int(use_graph))
    n = 0 if order is None else int(order.numel())
    reach = None
    if arm is not None:
        ik = ik if ik is not None else ik_params()
        reach = ScGenReach(ctypes.cast(ctypes.pointer(arm), P), ctypes.cast(ctypes.pointer(ik), P),
                           None if gate is None else gate.handle, None if rmap is None else rmap.handle)
    _check(lib().sc_generate(ctx.handle, ctypes.byref(db.c), ctypes.byref(p), _active_ptr(order), n,
                             None if cfg is None else ctypes.byref(cfg), None if reach is None else ctypes.byref(reach),
                             _ptr(poses), _ptr(valid), _ptr(band), _ptr(tries), _ptr(q_reach)))
    return poses, valid, band, tries


def ik_reach(ctx: Context, arm: ScArm, params: ScIkParams, targets: torch.Tensor, target_ids=None,
             with_band: bool = False):
    """sc_ik_reach. targets [n,12] f32 (device). Returns (reach u8 [n], q f32 [n,7], err f32 [n,2]),
    plus band u8 [n] if with_band."""
    dev = torch.device("cuda", ctx.device)
    n = targets.shape[0]
    reach = torch.empty(n, dtype=torch.uint8, device=dev)
    q = torch.empty((n, 7), dtype=torch.float32, device=dev)
    err = torch.empty((n, 2), dtype=torch.float32, device=dev)
    band = torch.empty(n, dtype=torch.uint8, device=dev) if with_band else None
    _check(lib().sc_ik_reach(ctx.handle, ctypes.byref(arm), ctypes.byref(params), _ptr(targets), _ptr(target_ids), n,
                             _ptr(reach), _ptr(q), _ptr(err), _ptr(band)))
    return (reach, q, err, band) if with_band else (reach, q, err)


def ik_dls_step(ctx: Context, arm: ScArm, lam: float, targets: torch.Tensor, q_in: torch.Tensor):
    """sc_ik_dls_step. Returns (q_out [n,7], tool [n,12] = FK of q_in)."""
    n = targets.shape[0]
    q_out = torch.empty_like(q_in)
    tool = torch.empty((n, 12), dtype=torch.float32, device=q_in.device)
    _check(lib().sc_ik_dls_step(ctx.handle, ctypes.byref(arm), lam, _ptr(targets), _ptr(q_in), n, _ptr(q_out),
                                _ptr(tool)))
    return q_out, tool


class Surrogate:
    """An sc_mlp handle (reachability gate)."""

    def __init__(self, ctx: Context, seed: int = 0, handle=None):
        self.ctx = ctx
        if handle is None:
            handle = P()
            _check(lib().sc_mlp_create(ctx.handle, seed, ctypes.byref(handle)))
        self.handle = handle

    @classmethod
    def load(cls, ctx: Context, path: str) -> "Surrogate":
        h = P()
        _check(lib().sc_mlp_load(ctx.handle, path.encode(), ctypes.byref(h)))
        return cls(ctx, handle=h)

    def save(self, path: str):
        _check(lib().sc_mlp_save(self.ctx.handle, self.handle, path.encode()))

    @staticmethod
    def param_count() -> int:
        return lib().sc_mlp_param_count()

    def get(self):
        """(params [134401] f32, mu [9], sigma [9], tau) as numpy."""
        n = self.param_count()
        p, mu, sd, tau = np.zeros(n, np.float32), np.zeros(9, np.float32), np.zeros(9, np.float32), ctypes.c_float()
        _check(lib().sc_mlp_get(self.ctx.handle, self.handle, _ptr(p), _ptr(mu), _ptr(sd), ctypes.byref(tau)))
        return p, mu, sd, tau.value

    def set(self, params=None, mu=None, sigma=None, tau=0.0):
        c = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
        p, m, s_ = c(params), c(mu), c(sigma)
        _check(lib().sc_mlp_set(self.ctx.handle, self.handle, _ptr(p), _ptr(m), _ptr(s_), float(tau)))

    def infer(self, targets: torch.Tensor) -> torch.Tensor:
        out = torch.empty(targets.shape[0], dtype=torch.float32, device=targets.device)
        _check(lib().sc_surrogate_infer(self.ctx.handle, self.handle, _ptr(targets), targets.shape[0], _ptr(out)))
        return out

    def grads(self, targets: torch.Tensor, labels: torch.Tensor):
        g = torch.empty(self.param_count(), dtype=torch.float32, device=targets.device)
        loss = ctypes.c_float()
        _check(lib().sc_surrogate_grads(self.ctx.handle, self.handle, _ptr(targets), _ptr(labels), targets.shape[0],
                                        _ptr(g), ctypes.byref(loss)))
        return g, loss.value

    def adam_step(self, grads: torch.Tensor | None, params: ScTrainParams):
        _check(lib().sc_mlp_adam_step(self.ctx.handle, self.handle, _ptr(grads), ctypes.byref(params)))

    def train_step(self, targets: torch.Tensor, labels: torch.Tensor, params: ScTrainParams) -> float:
        """One gradient + Adam step on the rows in order; returns the mean BCE."""
        loss = ctypes.c_float()
        _check(lib().sc_mlp_train_step(self.ctx.handle, self.handle, _ptr(targets), _ptr(labels), targets.shape[0],
                                       ctypes.byref(params), ctypes.byref(loss)))
        return loss.value

    def train(self, targets: torch.Tensor, labels: torch.Tensor, params: ScTrainParams):
        loss = np.zeros(max(1, params.epochs), np.float32)
        _check(lib().sc_surrogate_train(self.ctx.handle, self.handle, _ptr(targets), _ptr(labels), targets.shape[0],
                                        ctypes.byref(params), _ptr(loss)))
        return loss[: params.epochs]

    def tune_threshold(self, targets: torch.Tensor, labels: torch.Tensor, min_recall: float = 0.99):
        tau, rec, pr = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        _check(lib().sc_surrogate_tune_threshold(self.ctx.handle, self.handle, _ptr(targets), _ptr(labels),
                                                 targets.shape[0], float(min_recall), ctypes.byref(tau),
                                                 ctypes.byref(rec), ctypes.byref(pr)))
        return tau.value, rec.value, pr.value

    def close(self):
        if getattr(self, "handle", None):
            lib().sc_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


RMAP_DEFAULT = (64, 16, 64, -1.1, 1.5, 1.4)  # nz, nc, nxy, z_lo, z_hi, r_max: 4 cm cells around the arm


class ReachMap:
    """An sc_rmap handle: the 4D reachability map (RM4D-style) built from
    labelled IK outcomes; score >= tau passes."""

    def __init__(self, ctx: Context, params=RMAP_DEFAULT):
        self.ctx = ctx
        self.params = tuple(params)
        h = P()
        _check(lib().sc_rmap_create(ctx.handle, ctypes.byref(ScRmapParams(*params)), ctypes.byref(h)))
        self.handle = h
        self.tau = 1

    @property
    def cells(self) -> int:
        return lib().sc_rmap_cells(self.handle)

    def build(self, targets: torch.Tensor, labels: torch.Tensor):
        assert targets.dtype == torch.float32 and targets.is_contiguous() and targets.shape[1] == 12
        assert labels.dtype == torch.uint8 and labels.shape[0] == targets.shape[0]
        _check(lib().sc_rmap_build(self.ctx.handle, self.handle, _ptr(targets), _ptr(labels), targets.shape[0]))

    def query(self, targets: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        assert targets.dtype == torch.float32 and targets.is_contiguous() and targets.shape[1] == 12
        n = targets.shape[0]
        score = torch.empty(n, dtype=torch.uint16, device=targets.device) if out is None else out
        _check(lib().sc_rmap_query(self.ctx.handle, self.handle, _ptr(targets), n, _ptr(score)))
        return score

    def tune_threshold(self, targets: torch.Tensor, labels: torch.Tensor, min_recall: float = 0.99):
        tau, rec, pr = I32(), ctypes.c_float(), ctypes.c_float()
        _check(lib().sc_rmap_tune_threshold(self.ctx.handle, self.handle, _ptr(targets), _ptr(labels),
                                            targets.shape[0], float(min_recall), ctypes.byref(tau),
                                            ctypes.byref(rec), ctypes.byref(pr)))
        self.tau = tau.value
        return tau.value, rec.value, pr.value

    def set_threshold(self, tau: int):
        _check(lib().sc_rmap_set_threshold(self.handle, int(tau)))
        self.tau = int(tau)

    def counts(self) -> np.ndarray:
        """uint32 [cells][2] = (reachable, labels) per cell."""
        c = np.zeros((self.cells, 2), np.uint32)
        _check(lib().sc_rmap_get_counts(self.ctx.handle, self.handle, _ptr(c)))
        return c

    def close(self):
        if getattr(self, "handle", None):
            lib().sc_rmap_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sample_parts(ctx: Context, db: DeviceBatch, seed: int, active: torch.Tensor | None = None) -> torch.Tensor:
    """sc_sample_parts into the batch's joint-value array; returns it [n_cand][max_parts]."""
    if db.max_parts == 0:
        raise ValueError("the batch has no articulated parts")
    n = _n_items(db, active)
    _check(lib().sc_sample_parts(ctx.handle, ctypes.byref(db.c), seed, _active_ptr(active), n, _ptr(db.t["part_q"])))
    return db.part_q


def collide_last_work(ctx: Context):
    """(sphere pairs, sphere-box pairs) evaluated by the last collide call (synchronises)."""
    a, b = I64(), I64()
    _check(lib().sc_collide_last_work(ctx.handle, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ik_last_work(ctx: Context) -> int:
    """Seed-iterations (checks x seeds) of the last ik_reach call (synchronises)."""
    a = I64()
    _check(lib().sc_ik_last_work(ctx.handle, ctypes.byref(a)))
    return a.value


def collide_last_tri_work(ctx: Context) -> int:
    """Exact sphere-triangle distances of the last collide call (synchronises)."""
    a = I64()
    _check(lib().sc_collide_last_tri_work(ctx.handle, ctypes.byref(a)))
    return a.value


def order_by_work(batch) -> np.ndarray:
    """Candidate indices heaviest first (host helper sc_order_by_work)."""
    t = np.ascontiguousarray(batch.tmpl_obj_off, np.int32)
    o = np.ascontiguousarray(batch.obj_sph_off, np.int32)
    c = np.ascontiguousarray(batch.cand_tmpl_off, np.int32)
    out = np.empty(int(c[-1]), np.int32)
    _check(lib().sc_order_by_work(len(t) - 1, _ptr(t), _ptr(o), _ptr(c), _ptr(out)))
    return out
