"""FP64 CPU oracle for the Sceniris hot path (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference legs may import this package. It shares no code
with the CUDA library: it never imports ``paper_2512_16896_b300`` and is never
imported by it. Inputs are duck-typed scene batches (any object with the CSR
arrays documented in ``synth.SceneBatch``).

``sceniris_oracle.cpp`` holds the geometry, sampling, collision, generation
and IK definitions; ``mlp.py`` holds the surrogate network (numpy, FP64);
``rmap.py`` the 4D reachability map (cell keys in FP32, counts as integers).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sceniris_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2, no fast-math) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fno-fast-math", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lpthread"]
        subprocess.run(cmd, check=True)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


class _Scene(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("n_templates", "n_objects", "n_spheres", "n_verts", "n_obb", "n_cand")] + [
        (n, ctypes.c_void_p) for n in ("tmpl_obj_off", "obj_sph_off", "sph_local", "obj_half", "obj_rel",
                                       "obj_rel_param", "tmpl_poly_off", "poly_verts", "tmpl_support_z",
                                       "tmpl_obb_off", "obb", "cand_tmpl_off", "tmpl_base", "obj_rel_dir",
                                       "obj_anchor_off", "obj_anchor")] + [
        ("n_parts", ctypes.c_int32), ("max_parts", ctypes.c_int32)] + [
        (n, ctypes.c_void_p) for n in ("tmpl_part_off", "part_param", "obb_part", "part_q")] + [
        ("n_tri", ctypes.c_int32), ("tmpl_tri_off", ctypes.c_void_p), ("tri", ctypes.c_void_p)]


class _Arm(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float * 7) for n in ("dh_d", "dh_a", "dh_alpha", "qmin", "qmax")]


class _IkParams(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_float), ("tol_pos", ctypes.c_float), ("tol_rot", ctypes.c_float),
                ("iters", ctypes.c_int32), ("seeds", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class _GenParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("max_attempts", ctypes.c_int32), ("max_retries", ctypes.c_int32)]


def _declare(L):
    P = ctypes.c_void_p
    L.or_philox4x32_10.argtypes = [P, P, P]
    L.or_philox4x64_10.argtypes = [P, P, P]
    L.or_uniform4.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P]
    L.or_point_in_polygon.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
    L.or_point_in_polygon.restype = ctypes.c_int
    L.or_pose_offset.argtypes = [P, ctypes.c_int]
    L.or_pose_offset.restype = ctypes.c_int64
    L.or_sample_poses.argtypes = [P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                  ctypes.c_int, P, P, P, ctypes.c_int]
    L.or_sphere_world.argtypes = [P, P, P]
    L.or_sphere_sphere.argtypes = [P, P]
    L.or_sphere_sphere.restype = ctypes.c_double
    L.or_sphere_obb.argtypes = [P, P]
    L.or_sphere_obb.restype = ctypes.c_double
    L.or_collide.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int]
    L.or_fk_frames.argtypes = [P, P, P]
    L.or_jacobian.argtypes = [P, P, P]
    L.or_pose_error.argtypes = [P, P, P, P, P, P]
    L.or_dls_step.argtypes = [P, ctypes.c_double, P, P, P]
    L.or_ik_error.argtypes = [P, P, P, P, P]
    L.or_ik_seed.argtypes = [P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, P]
    L.or_ik_reach.argtypes = [P, P, P, P, ctypes.c_int, P, P, P, P, P, ctypes.c_int]
    L.or_grasp_target.argtypes = [P, ctypes.c_double, P, P]
    L.or_generate.argtypes = [P, P, P, P, P, ctypes.c_int, P, P, P, P, ctypes.c_int]
    L.or_sample_parts.argtypes = [P, ctypes.c_uint64, P, ctypes.c_int, P]
    L.or_point_triangle.argtypes = [P, P, P, P]
    L.or_point_triangle.restype = ctypes.c_double
    L.or_sphere_triangle.argtypes = [P, P]
    L.or_sphere_triangle.restype = ctypes.c_double


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def default_threads() -> int:
    return os.cpu_count() or 1


class Scene:
    """Holds contiguous copies of a batch's arrays and the C struct pointing at them."""

    def __init__(self, batch):
        self.keep = {
            "tmpl_obj_off": _c(batch.tmpl_obj_off, np.int32), "obj_sph_off": _c(batch.obj_sph_off, np.int32),
            "sph_local": _c(batch.sph_local, np.float32), "obj_half": _c(batch.obj_half, np.float32),
            "obj_rel": _c(batch.obj_rel, np.int32), "obj_rel_param": _c(batch.obj_rel_param, np.float32),
            "tmpl_poly_off": _c(batch.tmpl_poly_off, np.int32), "poly_verts": _c(batch.poly_verts, np.float32),
            "tmpl_support_z": _c(batch.tmpl_support_z, np.float32), "tmpl_obb_off": _c(batch.tmpl_obb_off, np.int32),
            "obb": _c(batch.obb, np.float32).reshape(-1, 12), "cand_tmpl_off": _c(batch.cand_tmpl_off, np.int32),
            "tmpl_base": _c(batch.tmpl_base, np.float32).reshape(-1, 4),
        }
        # optional relation arrays (None: no object uses them)
        for name, dt in (("obj_rel_dir", np.float32), ("obj_anchor_off", np.int32), ("obj_anchor", np.int32)):
            a = getattr(batch, name, None)
            self.keep[name] = None if a is None or np.asarray(a).size == 0 else _c(a, dt)
        if self.keep["obj_anchor"] is None:
            self.keep["obj_anchor_off"] = None
        # articulated parts and the candidates' joint values (None: no parts)
        self.max_parts = 0
        pp = getattr(batch, "part_param", None)
        if pp is not None and np.asarray(pp).size:
            self.keep["tmpl_part_off"] = _c(batch.tmpl_part_off, np.int32)
            self.keep["part_param"] = _c(pp, np.float32).reshape(-1, 12)
            op = getattr(batch, "obb_part", None)
            self.keep["obb_part"] = None if op is None or np.asarray(op).size == 0 else _c(op, np.int32)
            self.max_parts = int(np.diff(self.keep["tmpl_part_off"]).max())
            self.keep["part_q"] = _c(batch.part_q, np.float32).reshape(-1, self.max_parts)
            if len(self.keep["part_q"]) != int(self.keep["cand_tmpl_off"][-1]):
                raise ValueError("part_q needs one row of max_parts values per candidate")
        else:
            for name in ("tmpl_part_off", "part_param", "obb_part", "part_q"):
                self.keep[name] = None
        k = self.keep
        self.n_cand = int(k["cand_tmpl_off"][-1])
        self.c = _Scene(len(k["tmpl_obj_off"]) - 1, len(k["obj_half"]), len(k["sph_local"]), len(k["poly_verts"]),
                        len(k["obb"]), self.n_cand)
        # world meshes (None: no triangles)
        tr = getattr(batch, "tri", None)
        if tr is not None and np.asarray(tr).size:
            k["tmpl_tri_off"] = _c(batch.tmpl_tri_off, np.int32)
            k["tri"] = _c(tr, np.float32).reshape(-1, 12)
        else:
            k["tmpl_tri_off"] = k["tri"] = None
        for n, _ in _Scene._fields_[6:]:
            if n not in ("n_parts", "max_parts", "n_tri"):
                setattr(self.c, n, _ptr(k[n]))
        self.c.n_tri = 0 if k["tri"] is None else len(k["tri"])
        self.c.n_parts = 0 if k["part_param"] is None else len(k["part_param"])
        self.c.max_parts = self.max_parts
        sizes = np.diff(k["cand_tmpl_off"]).astype(np.int64) * np.diff(k["tmpl_obj_off"]).astype(np.int64)
        self.n_poses = int(sizes.sum())

    def ref(self):
        return ctypes.byref(self.c)


def philox4x32(ctr, key):
    c = _c(ctr, np.uint32); k = _c(key, np.uint32); o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def philox4x64(ctr, key):
    c = _c(ctr, np.uint64); k = _c(key, np.uint64); o = np.zeros(4, np.uint64)
    lib().or_philox4x64_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def uniform4(seed, cand, obj, retry, attempt):
    o = np.zeros(4, np.float64)
    lib().or_uniform4(seed, cand, obj, retry, attempt, _ptr(o))
    return o


def point_in_polygon(verts, p):
    v = np.asarray(verts, np.float64)
    vx, vy = _c(v[:, 0], np.float64), _c(v[:, 1], np.float64)
    d = np.zeros(1, np.float64)
    inside = lib().or_point_in_polygon(_ptr(vx), _ptr(vy), len(v), float(p[0]), float(p[1]), _ptr(d))
    return bool(inside), float(d[0])


def sphere_world(sph, pose):
    s = _c(sph, np.float32); p = _c(pose, np.float64); o = np.zeros(4)
    lib().or_sphere_world(_ptr(s), _ptr(p), _ptr(o))
    return o


def sphere_sphere(a, b):
    return lib().or_sphere_sphere(_ptr(_c(a, np.float64)), _ptr(_c(b, np.float64)))


def sphere_obb(sphere, box12):
    return lib().or_sphere_obb(_ptr(_c(sphere, np.float64)), _ptr(_c(box12, np.float32)))


def point_triangle(p, a, b, c):
    """Distance from point p to the filled triangle abc (FP64)."""
    return lib().or_point_triangle(*[_ptr(_c(x, np.float64)) for x in (p, a, b, c)])


def sphere_triangle(sphere, tri12):
    return lib().or_sphere_triangle(_ptr(_c(sphere, np.float64)), _ptr(_c(tri12, np.float32)))


def sample_poses(batch, seed, max_attempts=16, retry=0, first_obj=0, n_obj=1 << 30, active=None, poses=None,
                 threads=None):
    """Returns (poses [P,4] float64, ok [n] u8, band [n] u8) in the CSR pose layout."""
    sc = batch if isinstance(batch, Scene) else Scene(batch)
    poses = np.zeros((sc.n_poses, 4), np.float64) if poses is None else _c(poses, np.float64)
    act = None if active is None else _c(active, np.int32)
    n = sc.n_cand if act is None else len(act)
    ok = np.zeros(n, np.uint8); band = np.zeros(n, np.uint8)
    lib().or_sample_poses(sc.ref(), seed, max_attempts, retry, first_obj, n_obj, _ptr(act), n, _ptr(poses), _ptr(ok),
                          _ptr(band), threads or default_threads())
    return poses, ok, band


def sample_parts(batch, seed, active=None):
    """Joint values of every part of the listed candidates, float64
    [n_cand][max_parts] (entries of unlisted candidates and unused slots 0)."""
    sc = batch if isinstance(batch, Scene) else Scene(batch)
    if sc.max_parts == 0:
        raise ValueError("the batch has no articulated parts")
    q = np.zeros((sc.n_cand, sc.max_parts), np.float64)
    act = None if active is None else _c(active, np.int32)
    n = sc.n_cand if act is None else len(act)
    lib().or_sample_parts(sc.ref(), seed, _ptr(act), n, _ptr(q))
    return q


def collide(batch, poses, active=None, first_new=0, threads=None):
    """Returns (collide [n] u8, min_dist [n] float64, band [n] u8)."""
    sc = batch if isinstance(batch, Scene) else Scene(batch)
    p = _c(poses, np.float64)
    assert p.shape == (sc.n_poses, 4)
    act = None if active is None else _c(active, np.int32)
    n = sc.n_cand if act is None else len(act)
    col = np.zeros(n, np.uint8); md = np.zeros(n, np.float64); band = np.zeros(n, np.uint8)
    lib().or_collide(sc.ref(), _ptr(p), _ptr(act), n, first_new, _ptr(col), _ptr(md), _ptr(band),
                     threads or default_threads())
    return col, md, band


def make_arm(d, a, alpha, qmin, qmax):
    f = lambda v: (ctypes.c_float * 7)(*[float(x) for x in v])
    return _Arm(f(d), f(a), f(alpha), f(qmin), f(qmax))


def fk_frames(arm, q):
    o = np.zeros((8, 4, 4)); lib().or_fk_frames(ctypes.byref(arm), _ptr(_c(q, np.float64)), _ptr(o))
    return o


def jacobian(arm, q):
    o = np.zeros((6, 7)); lib().or_jacobian(ctypes.byref(arm), _ptr(_c(q, np.float64)), _ptr(o))
    return o


def pose_error(arm, q, target12):
    t = np.asarray(target12, np.float64)
    pe = np.zeros(1); re = np.zeros(1)
    lib().or_pose_error(ctypes.byref(arm), _ptr(_c(q, np.float64)), _ptr(_c(t[:9], np.float64)),
                        _ptr(_c(t[9:12], np.float64)), _ptr(pe), _ptr(re))
    return float(pe[0]), float(re[0])


def ik_error(arm, q, target12):
    t = np.asarray(target12, np.float64)
    e = np.zeros(6)
    lib().or_ik_error(ctypes.byref(arm), _ptr(_c(q, np.float64)), _ptr(_c(t[:9], np.float64)),
                      _ptr(_c(t[9:12], np.float64)), _ptr(e))
    return e


def dls_step(arm, lam, q, target12):
    t = np.asarray(target12, np.float64)
    q = _c(q, np.float64).copy()
    lib().or_dls_step(ctypes.byref(arm), float(lam), _ptr(_c(t[:9], np.float64)), _ptr(_c(t[9:12], np.float64)),
                      _ptr(q))
    return q


def ik_params(lam=0.05, tol_pos=5e-3, tol_rot=0.05, iters=100, seeds=32, seed=3):
    return _IkParams(lam, tol_pos, tol_rot, iters, seeds, seed)


def ik_seed(arm, seed, target, s):
    q = np.zeros(7); lib().or_ik_seed(ctypes.byref(arm), seed, target, s, _ptr(q))
    return q


def ik_reach(arm, params, targets, target_ids=None, threads=None, with_band=False):
    """Returns (reach [n] u8, q [n,7], err [n,2], iters [n]), plus band [n] u8
    (a success check of some seed within 1e-5 of a tolerance) if with_band."""
    t = _c(targets, np.float32).reshape(-1, 12)
    n = len(t)
    ids = None if target_ids is None else _c(target_ids, np.uint32)
    reach = np.zeros(n, np.uint8); q = np.zeros((n, 7)); err = np.zeros((n, 2)); it = np.zeros(n, np.int32)
    band = np.zeros(n, np.uint8)
    lib().or_ik_reach(ctypes.byref(arm), ctypes.byref(params), _ptr(t), _ptr(ids), n, _ptr(reach), _ptr(q), _ptr(err),
                      _ptr(it), _ptr(band), threads or default_threads())
    return (reach, q, err, it, band) if with_band else (reach, q, err, it)


def grasp_target(pose, hz, base):
    o = np.zeros(12)
    lib().or_grasp_target(_ptr(_c(pose, np.float64)), float(hz), _ptr(_c(base, np.float32)), _ptr(o))
    return o


def generate(batch, seed, max_attempts=16, max_retries=10, arm=None, ikp=None, active=None, threads=None):
    """Returns (poses [P,4] float64, valid [n] u8, band [n] u8, tries [n] int32)."""
    sc = batch if isinstance(batch, Scene) else Scene(batch)
    g = _GenParams(seed, max_attempts, max_retries)
    act = None if active is None else _c(active, np.int32)
    n = sc.n_cand if act is None else len(act)
    poses = np.full((sc.n_poses, 4), np.nan)
    valid = np.zeros(n, np.uint8); band = np.zeros(n, np.uint8); tries = np.zeros(n, np.int32)
    lib().or_generate(sc.ref(), ctypes.byref(g), None if arm is None else ctypes.byref(arm),
                      None if ikp is None else ctypes.byref(ikp), _ptr(act), n, _ptr(poses), _ptr(valid), _ptr(band),
                      _ptr(tries), threads or default_threads())
    return poses, valid, band, tries


def pose_offsets(batch):
    """CSR pose offset of every candidate, computed by the oracle's own loop."""
    sc = batch if isinstance(batch, Scene) else Scene(batch)
    return np.array([lib().or_pose_offset(sc.ref(), c) for c in range(sc.n_cand)], np.int64)
