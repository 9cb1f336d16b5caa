"""Seeded synthetic inputs shared by the GPU library's tests/bench and the oracle.

This module only *draws* inputs: template geometry (collision spheres, support
polygons, static-world boxes, relation graphs), IK target poses and MLP
training inputs. It holds none of the method's arithmetic (no sampling of
poses, no distances, no kinematics). Every array is plain numpy so the same
object feeds the FP64 oracle and the CUDA library.

The paper's benchmark scenes are built from its own mesh assets (an apple, a
banana in a drawer, a cabinet; Sec. V-A), which are not available; the shapes
below stand in for them with the sizes of the tabletop/shelf workloads:

  * tabletop:  1 template, 1.2 x 0.8 m table at z = 0.75, 8 objects x 16 spheres,
               all free, B = 1024 candidates (seed 0).
  * shelf:     1 template, 32 objects x 64 spheres, 25% on-top / 25% next-to /
               50% free, 20 random OBBs, B = 65,536 (seed 1).
  * ragged:    4096 templates, 4..64 objects, 8..128 spheres per object, convex
               4..10-gon supports of area 0.5..2 m^2, 64 candidates each (seed 2).

Object assets: sphere centres uniform in a local box of per-axis half extent
U(0.05, 0.15) m, radii U(0.01, 0.05) m; the object frame is then moved to the
centre of the spheres' tight axis-aligned bounding box, whose half extents
(Hx, Hy, Hz) and xy bounding radius rho are part of the asset description.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

REL_FREE, REL_ON_TOP, REL_NEXT_TO, REL_DIRECTIONAL, REL_MIDDLE, REL_INSIDE = 0, 1, 2, 3, 4, 5
REL_REACH, REL_LOCAL, REL_FACE_TO = 0x10, 0x20, 0x40

# 7-DoF arm used by the reachability workload: standard DH parameters.
ARM_D = (0.333, 0.0, 0.316, 0.0, 0.384, 0.0, 0.107)
ARM_A = (0.0, 0.0, 0.0, 0.0825, -0.0825, 0.0, 0.088)
ARM_ALPHA = (0.0, -math.pi / 2, math.pi / 2, math.pi / 2, -math.pi / 2, math.pi / 2, math.pi / 2)
ARM_QLIM = 2.8


@dataclasses.dataclass
class SceneBatch:
    """CSR-packed scene templates plus candidate ranges (host numpy arrays).

    Layouts (all little-endian, C-contiguous):
      tmpl_obj_off  int32 [T+1]  objects of template t are [off[t], off[t+1])
      obj_sph_off   int32 [O+1]  spheres of object o
      sph_local     f32 [S,4]    (x, y, z, r) in the object frame
      obj_half      f32 [O,4]    (Hx, Hy, Hz, rho_xy)
      obj_rel       int32 [O]    kind | flags (REL_REACH, REL_LOCAL, REL_FACE_TO) | (reference local index << 8)
      obj_rel_param f32 [O,4]    (dmin, dmax, ratio_on_support, 0); directional: (min_r, max_r, ratio, theta)
      obj_rel_dir   f32 [O]      direction angle of a directional relation (radians)
      obj_anchor_off int32 [O+1]; obj_anchor int32 [A]: anchors (local indices) of a middle relation
      tmpl_poly_off int32 [T+1]; poly_verts f32 [V,2] (CCW)
      tmpl_support_z f32 [T]
      tmpl_obb_off  int32 [T+1]; obb f32 [n_obb,12] centre(x,y,z,0) quat(x,y,z,w) half(x,y,z,0)
      cand_tmpl_off int32 [T+1]  candidates of template t
      tmpl_base     f32 [T,4]    robot base (x, y, z, yaw)
      tmpl_part_off int32 [T+1]; part_param f32 [n_parts,12]: articulated (prismatic) parts,
                                 (axis, qmin), (qmax, support centre), (support half x, y, yaw, 0)
      obb_part      int32 [n_obb] template-local part a box moves with (-1: static)
      part_q        f32 [B, max_parts] joint value of every part per candidate (drawn here)
      tmpl_tri_off  int32 [T+1]; tri f32 [n_tri,12]: world mesh triangles a | b | c (x, y, z, 0)
    """

    tmpl_obj_off: np.ndarray
    obj_sph_off: np.ndarray
    sph_local: np.ndarray
    obj_half: np.ndarray
    obj_rel: np.ndarray
    obj_rel_param: np.ndarray
    tmpl_poly_off: np.ndarray
    poly_verts: np.ndarray
    tmpl_support_z: np.ndarray
    tmpl_obb_off: np.ndarray
    obb: np.ndarray
    cand_tmpl_off: np.ndarray
    tmpl_base: np.ndarray
    obj_rel_dir: np.ndarray = None
    obj_anchor_off: np.ndarray = None
    obj_anchor: np.ndarray = None
    tmpl_part_off: np.ndarray = None
    part_param: np.ndarray = None
    obb_part: np.ndarray = None
    part_q: np.ndarray = None
    tmpl_tri_off: np.ndarray = None
    tri: np.ndarray = None
    name: str = ""

    @property
    def n_templates(self) -> int:
        return len(self.tmpl_obj_off) - 1

    @property
    def n_objects(self) -> int:
        return len(self.obj_half)

    @property
    def n_spheres(self) -> int:
        return len(self.sph_local)

    @property
    def n_cand(self) -> int:
        return int(self.cand_tmpl_off[-1])

    def n_obj_of(self, t: int) -> int:
        return int(self.tmpl_obj_off[t + 1] - self.tmpl_obj_off[t])

    def cand_template(self) -> np.ndarray:
        """Template index of every candidate (int32 [B])."""
        counts = np.diff(self.cand_tmpl_off)
        return np.repeat(np.arange(self.n_templates, dtype=np.int32), counts)

    def tmpl_pose_off(self) -> np.ndarray:
        """Start of each template's block in the CSR pose array (int64 [T+1]):
        template t holds n_cand(t) x n_obj(t) poses, candidate-major."""
        sizes = np.diff(self.cand_tmpl_off).astype(np.int64) * np.diff(self.tmpl_obj_off).astype(np.int64)
        return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    def n_poses(self) -> int:
        return int(self.tmpl_pose_off()[-1])

    def sphere_count_of_template(self) -> np.ndarray:
        return (self.obj_sph_off[self.tmpl_obj_off[1:]] - self.obj_sph_off[self.tmpl_obj_off[:-1]]).astype(np.int64)

    def subset(self, templates) -> "SceneBatch":
        """A batch made of the listed templates (their candidates keep their count)."""
        templates = list(templates)
        parts = []
        for t in templates:
            o0, o1 = int(self.tmpl_obj_off[t]), int(self.tmpl_obj_off[t + 1])
            s0, s1 = int(self.obj_sph_off[o0]), int(self.obj_sph_off[o1])
            v0, v1 = int(self.tmpl_poly_off[t]), int(self.tmpl_poly_off[t + 1])
            b0, b1 = int(self.tmpl_obb_off[t]), int(self.tmpl_obb_off[t + 1])
            anchors = [list(self.obj_anchor[self.obj_anchor_off[o]:self.obj_anchor_off[o + 1]]) for o in range(o0, o1)]
            extra = {}
            if self.part_param is not None:
                p0, p1 = int(self.tmpl_part_off[t]), int(self.tmpl_part_off[t + 1])
                c0, c1 = int(self.cand_tmpl_off[t]), int(self.cand_tmpl_off[t + 1])
                extra = dict(parts=self.part_param[p0:p1], obb_part=self.obb_part[b0:b1],
                             part_q=self.part_q[c0:c1, :p1 - p0])
            if self.tri is not None:
                extra["tri"] = self.tri[int(self.tmpl_tri_off[t]):int(self.tmpl_tri_off[t + 1])]
            parts.append(dict(**extra,
                sph=self.sph_local[s0:s1], nsph=np.diff(self.obj_sph_off[o0:o1 + 1]),
                half=self.obj_half[o0:o1], rel=self.obj_rel[o0:o1], relp=self.obj_rel_param[o0:o1],
                dir=self.obj_rel_dir[o0:o1], anchors=anchors,
                poly=self.poly_verts[v0:v1], z=self.tmpl_support_z[t], obb=self.obb[b0:b1],
                ncand=int(self.cand_tmpl_off[t + 1] - self.cand_tmpl_off[t]), base=self.tmpl_base[t]))
        return _pack(parts, name=f"{self.name}[subset {len(templates)}]")


def _pack(parts, name="") -> SceneBatch:
    def off(counts):
        return np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)

    nobj = [len(p["half"]) for p in parts]
    nsph = np.concatenate([p["nsph"] for p in parts]).astype(np.int64)
    anchors = [list(a) for p in parts for a in p.get("anchors", [[]] * len(p["half"]))]
    return SceneBatch(
        tmpl_obj_off=off(nobj),
        obj_sph_off=off(nsph),
        sph_local=np.ascontiguousarray(np.concatenate([p["sph"] for p in parts]).astype(np.float32)),
        obj_half=np.ascontiguousarray(np.concatenate([p["half"] for p in parts]).astype(np.float32)),
        obj_rel=np.ascontiguousarray(np.concatenate([p["rel"] for p in parts]).astype(np.int32)),
        obj_rel_param=np.ascontiguousarray(np.concatenate([p["relp"] for p in parts]).astype(np.float32)),
        tmpl_poly_off=off([len(p["poly"]) for p in parts]),
        poly_verts=np.ascontiguousarray(np.concatenate([p["poly"] for p in parts]).astype(np.float32)),
        tmpl_support_z=np.array([p["z"] for p in parts], dtype=np.float32),
        tmpl_obb_off=off([len(p["obb"]) for p in parts]),
        obb=np.ascontiguousarray(np.concatenate([p["obb"] for p in parts]).astype(np.float32).reshape(-1, 12)),
        cand_tmpl_off=off([p["ncand"] for p in parts]),
        tmpl_base=np.ascontiguousarray(np.array([p["base"] for p in parts], dtype=np.float32).reshape(-1, 4)),
        obj_rel_dir=np.ascontiguousarray(np.concatenate([p.get("dir", np.zeros(len(p["half"]))) for p in parts])
                                         .astype(np.float32)),
        obj_anchor_off=off([len(a) for a in anchors]),
        obj_anchor=np.array([i for a in anchors for i in a], dtype=np.int32),
        name=name,
        **_pack_parts(parts),
        **_pack_meshes(parts),
    )


def _pack_meshes(parts) -> dict:
    """CSR arrays of the world triangles (empty dict when no template has any)."""
    if not any(len(p.get("tri", ())) for p in parts):
        return {}
    tris = [np.asarray(p.get("tri", np.zeros((0, 12))), np.float32).reshape(-1, 12) for p in parts]
    return dict(tmpl_tri_off=np.concatenate([[0], np.cumsum([len(t) for t in tris])]).astype(np.int32),
                tri=np.ascontiguousarray(np.concatenate(tris)))


def _pack_parts(parts) -> dict:
    """CSR arrays of the articulated parts (empty dict when no template has any)."""
    if not any(len(p.get("parts", ())) for p in parts):
        return {}
    n_parts = [len(p.get("parts", ())) for p in parts]
    max_parts = max(n_parts)
    q = np.zeros((sum(p["ncand"] for p in parts), max_parts), np.float32)
    row = 0
    for p, n in zip(parts, n_parts):
        if n:
            q[row:row + p["ncand"], :n] = p["part_q"]
        row += p["ncand"]
    return dict(
        tmpl_part_off=np.concatenate([[0], np.cumsum(n_parts)]).astype(np.int32),
        part_param=np.ascontiguousarray(np.concatenate([np.asarray(p.get("parts", np.zeros((0, 12))), np.float32)
                                                        .reshape(-1, 12) for p in parts])),
        obb_part=np.concatenate([np.asarray(p.get("obb_part", -np.ones(len(p["obb"]))), np.int32)
                                 for p in parts]).astype(np.int32),
        part_q=q,
    )


def draw_object(rng: np.random.Generator, n_spheres: int, h_range=(0.05, 0.15), r_range=(0.01, 0.05)):
    """One object asset: (spheres [n,4] in the AABB-centred frame, half extents (Hx,Hy,Hz), rho)."""
    h = rng.uniform(h_range[0], h_range[1], size=3)
    c = rng.uniform(-h, h, size=(n_spheres, 3))
    r = rng.uniform(r_range[0], r_range[1], size=n_spheres)
    lo = (c - r[:, None]).min(axis=0)
    hi = (c + r[:, None]).max(axis=0)
    centre = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo)
    c = c - centre
    # asset description: xy bounding radius of the sphere set in its own frame
    rho = float(np.max(np.hypot(c[:, 0], c[:, 1]) + r))
    sph = np.concatenate([c, r[:, None]], axis=1).astype(np.float32)
    return sph, half.astype(np.float32), np.float32(rho)


def draw_relations(rng: np.random.Generator, n: int, n_reach: int = 0):
    """Relation kinds and reference objects: object 0 free; round(n/4) on-top and
    round(n/4) next-to objects chosen by a random permutation of 1..n-1; each
    refers to a uniformly random earlier object. The first n_reach objects carry
    the reachability flag."""
    kinds = np.zeros(n, dtype=np.int32)
    refs = np.zeros(n, dtype=np.int32)
    q = int(math.floor(0.25 * n + 0.5))
    perm = rng.permutation(np.arange(1, n))
    kinds[perm[:q]] = REL_ON_TOP
    kinds[perm[q:2 * q]] = REL_NEXT_TO
    for k in range(1, n):
        if kinds[k] != REL_FREE:
            refs[k] = rng.integers(0, k)
    rel = kinds | (refs << 8)
    rel[: min(n_reach, n)] |= REL_REACH
    return rel.astype(np.int32)


def draw_relations_hard(rng: np.random.Generator, n: int, n_reach: int = 0):
    """The full relation set of Sec. IV-F: object 0 free; of objects 1..n-1
    (random permutation) about 15% on-top, 15% next-to, 30% directional
    (one anchor: a partial annulus around it, direction +-x / +-y or a random
    angle, in the world or the anchor's frame, half-angle pi/8, pi/4 or pi/2,
    distance 'greater' [d, inf), 'less' [0, d] or 'equal' [d - 0.02, d + 0.02]
    with d ~ U(0.2, 0.6) m measured between positions), 15% middle (2 to 4
    earlier anchors) and the rest free; a quarter of the non-on-top objects
    face a random earlier object. Returns (rel, relp, dir, anchors)."""
    kinds = np.zeros(n, dtype=np.int32)
    refs = np.zeros(n, dtype=np.int32)
    relp = np.tile(np.array([0.05, 0.2, 0.0, 0.0], dtype=np.float32), (n, 1))
    dirs = np.zeros(n, dtype=np.float32)
    flags = np.zeros(n, dtype=np.int32)
    anchors = [[] for _ in range(n)]
    perm = rng.permutation(np.arange(1, n))
    m = len(perm)
    cut = np.cumsum([int(round(f * m)) for f in (0.15, 0.15, 0.30, 0.15)])
    kinds[perm[:cut[0]]] = REL_ON_TOP
    kinds[perm[cut[0]:cut[1]]] = REL_NEXT_TO
    kinds[perm[cut[1]:cut[2]]] = REL_DIRECTIONAL
    kinds[perm[cut[2]:cut[3]]] = REL_MIDDLE
    for k in range(1, n):
        refs[k] = rng.integers(0, k)
        if kinds[k] == REL_DIRECTIONAL:
            choice = rng.integers(0, 5)
            dirs[k] = [0.0, math.pi, 0.5 * math.pi, -0.5 * math.pi, 0.0][choice]
            if choice == 4:
                dirs[k] = rng.uniform(-math.pi, math.pi)
            if rng.uniform() < 0.5:
                flags[k] |= REL_LOCAL
            theta = [math.pi / 8, math.pi / 4, math.pi / 2][rng.integers(0, 3)]
            d = rng.uniform(0.2, 0.6)
            dt = rng.integers(0, 3)
            lo, hi = [(d, math.inf), (0.0, d), (d - 0.02, d + 0.02)][dt]
            relp[k] = [lo, hi, 0.0, theta]
        elif kinds[k] == REL_MIDDLE:
            na = min(k, int(rng.integers(2, 5)))
            if na < 2:
                kinds[k] = REL_FREE
            else:
                anchors[k] = sorted(rng.choice(k, size=na, replace=False).tolist())
                refs[k] = anchors[k][0]
        if kinds[k] != REL_ON_TOP and rng.uniform() < 0.25:
            flags[k] |= REL_FACE_TO
    rel = kinds | flags | (refs << 8)
    rel[: min(n_reach, n)] |= REL_REACH
    return rel.astype(np.int32), relp, dirs, anchors


def rect_polygon(lx: float, ly: float) -> np.ndarray:
    return np.array([[-lx / 2, -ly / 2], [lx / 2, -ly / 2], [lx / 2, ly / 2], [-lx / 2, ly / 2]], dtype=np.float32)


def convex_polygon(rng: np.random.Generator, n_verts: int, area: float) -> np.ndarray:
    """Convex CCW n-gon: sorted uniform angles on the unit circle, scaled to `area`."""
    ang = np.sort(rng.uniform(0.0, 2 * math.pi, size=n_verts))
    v = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    x, y = v[:, 0], v[:, 1]
    a0 = 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))
    return (v * math.sqrt(area / a0)).astype(np.float32)


def random_obbs(rng: np.random.Generator, n: int) -> np.ndarray:
    """Shelf-like static world: centres uniform in [-1.2,1.2]x[-1,1]x[0,2] m,
    uniformly random rotations (Shoemake's subgroup algorithm), sides U(0.02, 1.0) m."""
    out = np.zeros((n, 12), dtype=np.float64)
    out[:, 0] = rng.uniform(-1.2, 1.2, n)
    out[:, 1] = rng.uniform(-1.0, 1.0, n)
    out[:, 2] = rng.uniform(0.0, 2.0, n)
    u1, u2, u3 = rng.uniform(size=(3, n))
    out[:, 4] = np.sqrt(1 - u1) * np.sin(2 * math.pi * u2)
    out[:, 5] = np.sqrt(1 - u1) * np.cos(2 * math.pi * u2)
    out[:, 6] = np.sqrt(u1) * np.sin(2 * math.pi * u3)
    out[:, 7] = np.sqrt(u1) * np.cos(2 * math.pi * u3)
    out[:, 8:11] = 0.5 * rng.uniform(0.02, 1.0, size=(n, 3))
    return out.astype(np.float32)


def make_template(rng, n_obj, sph_counts, poly, support_z=0.75, n_obb=0, relations=True, n_reach=0,
                  ratio_on_support=0.0, base=None):
    sph, nsph, half = [], [], []
    for k in range(n_obj):
        s, h, rho = draw_object(rng, int(sph_counts[k]))
        sph.append(s)
        nsph.append(len(s))
        half.append([h[0], h[1], h[2], rho])
    dirs = np.zeros(n_obj, dtype=np.float32)
    anchors = [[] for _ in range(n_obj)]
    relp = np.tile(np.array([0.05, 0.2, ratio_on_support, 0.0], dtype=np.float32), (n_obj, 1))
    if relations == "hard":
        rel, relp, dirs, anchors = draw_relations_hard(rng, n_obj, n_reach)
        relp[:, 2] = ratio_on_support
    elif relations:
        rel = draw_relations(rng, n_obj, n_reach)
    else:
        rel = np.zeros(n_obj, dtype=np.int32)
        rel[: min(n_reach, n_obj)] |= REL_REACH
    obb = random_obbs(rng, n_obb) if n_obb else np.zeros((0, 12), np.float32)
    if base is None:  # robot at the middle of the support's -x side, facing +x
        base = [float(poly[:, 0].min()), 0.0, support_z, 0.0]
    return dict(sph=np.concatenate(sph), nsph=np.array(nsph), half=np.array(half, np.float32), rel=rel, relp=relp,
                dir=dirs, anchors=anchors, poly=poly, z=support_z, obb=obb, base=np.array(base, np.float32))


def tabletop(seed: int = 0, n_cand: int = 1024, n_obj: int = 8, n_sph: int = 16) -> SceneBatch:
    """Small tabletop workload: 1.2 x 0.8 m table, 8 free objects x 16 spheres."""
    rng = np.random.default_rng(seed)
    p = make_template(rng, n_obj, [n_sph] * n_obj, rect_polygon(1.2, 0.8), relations=False, n_reach=4,
                      base=[-0.6, 0.0, 0.75, 0.0])
    p["ncand"] = n_cand
    return _pack([p], name=f"tabletop {n_obj}x{n_sph} B={n_cand}")


def shelf(seed: int = 1, n_cand: int = 65536, n_obj: int = 32, n_sph: int = 64, n_obb: int = 20) -> SceneBatch:
    """Shelf workload: 32 objects x 64 spheres with relations, 20 random OBBs."""
    rng = np.random.default_rng(seed)
    p = make_template(rng, n_obj, [n_sph] * n_obj, rect_polygon(1.2, 0.8), n_obb=n_obb, n_reach=4,
                      base=[-0.6, 0.0, 0.75, 0.0])
    p["ncand"] = n_cand
    return _pack([p], name=f"shelf {n_obj}x{n_sph} obb={n_obb} B={n_cand}")


def ragged(seed: int = 2, n_templates: int = 4096, cand_per_template: int = 64, obj_range=(4, 64),
           sph_range=(8, 128), n_reach: int = 4) -> SceneBatch:
    """Ragged workload: many templates with uneven object and sphere counts."""
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_templates):
        n = int(rng.integers(obj_range[0], obj_range[1] + 1))
        counts = rng.integers(sph_range[0], sph_range[1] + 1, size=n)
        poly = convex_polygon(rng, int(rng.integers(4, 11)), float(rng.uniform(0.5, 2.0)))
        p = make_template(rng, n, counts, poly, n_reach=n_reach)
        p["ncand"] = cand_per_template
        parts.append(p)
    return _pack(parts, name=f"ragged T={n_templates}x{cand_per_template}")


def hard(seed: int = 5, n_templates: int = 256, cand_per_template: int = 64, obj_range=(6, 24),
         sph_range=(8, 64), n_reach: int = 0) -> SceneBatch:
    """Relation-heavy workload, a stand-in for the paper's harder benchmark
    scenes (Sec. V-A): every template uses the full relation set
    (draw_relations_hard) on a convex 4..10-gon support of area 1..3 m^2."""
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_templates):
        n = int(rng.integers(obj_range[0], obj_range[1] + 1))
        counts = rng.integers(sph_range[0], sph_range[1] + 1, size=n)
        poly = convex_polygon(rng, int(rng.integers(4, 11)), float(rng.uniform(1.0, 3.0)))
        p = make_template(rng, n, counts, poly, relations="hard", n_reach=n_reach)
        p["ncand"] = cand_per_template
        parts.append(p)
    return _pack(parts, name=f"hard T={n_templates}x{cand_per_template}")


def _box(c, h):
    """One axis-aligned world box row: centre c, identity quaternion, half extents h."""
    return [c[0], c[1], c[2], 0.0, 0.0, 0.0, 0.0, 1.0, h[0], h[1], h[2], 0.0]


def cabinet_template(rng, n_counter, n_drawers, inside_per_drawer, n_sph, q_max=0.35, counter_z=0.9):
    """A kitchen counter over a column of drawers (stand-in for the paper's
    cabinet with drawers, Sec. V-A). Counter: a 0.6 x 1.6 m support at
    z = counter_z with n_counter objects related as in draw_relations, its
    plate 1 mm below. Static carcass: the plate, two side panels and a back
    panel. Drawer j (prismatic, axis -x, q in [0, q_max]): floor plane at
    z = 0.04 + 0.28 j, inside support 0.49 x 0.55 m centred on the cabinet's
    axis at q = 0, a floor box 1 mm below it and four 13 cm walls 1 cm thick
    (5 boxes that move with the drawer). After the counter objects,
    inside_per_drawer objects per drawer with the INSIDE relation (erosion
    ratio 1), smaller assets (half extents U(0.03, 0.07), radii U(0.01, 0.03)).
    Joint values of the candidates are drawn later (uniform in the range)."""
    p = make_template(rng, n_counter, [n_sph] * n_counter, rect_polygon(0.6, 1.6), support_z=counter_z,
                      base=[-0.9, 0.0, counter_z, 0.0])
    obb = [_box((0.0, 0.0, counter_z - 0.016), (0.3, 0.8, 0.015)),
           _box((0.0, 0.31, 0.44), (0.3, 0.01, 0.42)), _box((0.0, -0.31, 0.44), (0.3, 0.01, 0.42)),
           _box((0.29, 0.0, 0.44), (0.01, 0.3, 0.42))]
    obb_part = [-1] * len(obb)
    parts = []
    for j in range(n_drawers):
        zf = 0.04 + 0.28 * j
        parts.append([-1.0, 0.0, 0.0, 0.0, q_max, 0.0, 0.0, zf, 0.245, 0.275, 0.0, 0.0])
        obb += [_box((0.0, 0.0, zf - 0.006), (0.26, 0.29, 0.005)),
                _box((-0.255, 0.0, zf + 0.06), (0.005, 0.29, 0.065)), _box((0.255, 0.0, zf + 0.06), (0.005, 0.29, 0.065)),
                _box((0.0, 0.285, zf + 0.06), (0.25, 0.005, 0.065)), _box((0.0, -0.285, zf + 0.06), (0.25, 0.005, 0.065))]
        obb_part += [j] * 5
    sph, nsph, half, rel, relp = [p["sph"]], list(p["nsph"]), list(p["half"]), list(p["rel"]), list(p["relp"])
    for j in range(n_drawers):
        for _ in range(inside_per_drawer):
            s, h, rho = draw_object(rng, n_sph, h_range=(0.03, 0.07), r_range=(0.01, 0.03))
            sph.append(s)
            nsph.append(len(s))
            half.append([h[0], h[1], h[2], rho])
            rel.append(REL_INSIDE | (j << 8))
            relp.append([0.0, 0.0, 1.0, 0.0])
    n = len(half)
    p.update(sph=np.concatenate(sph), nsph=np.array(nsph), half=np.array(half, np.float32),
             rel=np.array(rel, np.int32), relp=np.array(relp, np.float32), dir=np.zeros(n, np.float32),
             anchors=[[] for _ in range(n)], obb=np.array(obb, np.float32), obb_part=np.array(obb_part, np.int32),
             parts=np.array(parts, np.float32))
    return p


def cabinet(seed: int = 6, n_templates: int = 64, cand_per_template: int = 64, counter_range=(4, 10),
            drawer_range=(2, 3), inside_per_drawer: int = 2, n_sph: int = 16) -> SceneBatch:
    """Articulated workload: cabinet_template with 2..3 drawers and 4..10
    counter objects per template; every candidate draws each drawer's joint
    value uniformly in its range (seeded numpy, the same values for the
    library and the oracle)."""
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_templates):
        nd = int(rng.integers(drawer_range[0], drawer_range[1] + 1))
        nc = int(rng.integers(counter_range[0], counter_range[1] + 1))
        p = cabinet_template(rng, nc, nd, inside_per_drawer, n_sph)
        p["ncand"] = cand_per_template
        lo, hi = p["parts"][:, 3], p["parts"][:, 4]
        p["part_q"] = (lo + (hi - lo) * rng.uniform(size=(cand_per_template, nd))).astype(np.float32)
        parts.append(p)
    return _pack(parts, name=f"cabinet T={n_templates}x{cand_per_template}")


def _tri_rows(v, faces):
    """Triangle rows (a, 0, b, 0, c, 0) of faces [m,3] over vertices v [n,3]."""
    out = np.zeros((len(faces), 12), np.float64)
    for i in range(3):
        out[:, 4 * i:4 * i + 3] = v[np.asarray(faces)[:, i]]
    return out


def box_mesh(centre, rot, half):
    """The 12 triangles of a box surface: half extents `half`, rotation matrix
    `rot` (3x3), centre `centre`."""
    s = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float64)
    v = (s * np.asarray(half)) @ np.asarray(rot).T + np.asarray(centre)
    faces = [(0, 1, 3), (0, 3, 2), (4, 6, 7), (4, 7, 5), (0, 4, 5), (0, 5, 1),
             (2, 3, 7), (2, 7, 6), (0, 2, 6), (0, 6, 4), (1, 5, 7), (1, 7, 3)]
    return _tri_rows(v, faces)


def sphere_mesh(centre, radius, n_lat=8, n_lon=12):
    """A latitude-longitude sphere surface: 2 n_lon (n_lat - 1) triangles."""
    v = [[0.0, 0.0, 1.0]]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2 * math.pi * j / n_lon
            v.append([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    v.append([0.0, 0.0, -1.0])
    v = np.array(v) * radius + np.asarray(centre)
    ring = lambda i, j: 1 + (i - 1) * n_lon + (j % n_lon)
    faces = [(0, ring(1, j), ring(1, j + 1)) for j in range(n_lon)]
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            faces += [(ring(i, j), ring(i + 1, j), ring(i + 1, j + 1)), (ring(i, j), ring(i + 1, j + 1), ring(i, j + 1))]
    last = len(v) - 1
    faces += [(last, ring(n_lat - 1, j + 1), ring(n_lat - 1, j)) for j in range(n_lon)]
    return _tri_rows(v, faces)


def _rot_z_tilt(rng):
    """A random rotation: yaw U(0, 2 pi) then a tilt U(-0.3, 0.3) rad about x."""
    a, b = rng.uniform(0, 2 * math.pi), rng.uniform(-0.3, 0.3)
    rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    return rz @ rx


def meshes(seed: int = 7, n_templates: int = 4096, cand_per_template: int = 64, obj_range=(4, 24),
           sph_range=(8, 64), box_range=(2, 6), ball_range=(1, 3)) -> SceneBatch:
    """World-mesh workload (stand-in for the paper's mesh worlds checked by
    cuRobo, Sec. IV-D): the ragged recipe's objects (relations as in
    draw_relations) on convex 4..10-gon supports of 1..3 m^2 at z = 0.75,
    cluttered by U{2..6} box meshes (12 triangles; half extents U(0.03, 0.25),
    a random yaw and a tilt within 0.3 rad) and U{1..3} sphere meshes
    (192 triangles, radius U(0.05, 0.2)), centres uniform over the support's
    bounding box at heights U(0.70, 1.10)."""
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_templates):
        n = int(rng.integers(obj_range[0], obj_range[1] + 1))
        counts = rng.integers(sph_range[0], sph_range[1] + 1, size=n)
        poly = convex_polygon(rng, int(rng.integers(4, 11)), float(rng.uniform(1.0, 3.0)))
        p = make_template(rng, n, counts, poly)
        lo, hi = poly.min(axis=0), poly.max(axis=0)
        tris = []
        for _ in range(int(rng.integers(box_range[0], box_range[1] + 1))):
            c = [rng.uniform(lo[0], hi[0]), rng.uniform(lo[1], hi[1]), rng.uniform(0.70, 1.10)]
            tris.append(box_mesh(c, _rot_z_tilt(rng), rng.uniform(0.03, 0.25, 3)))
        for _ in range(int(rng.integers(ball_range[0], ball_range[1] + 1))):
            c = [rng.uniform(lo[0], hi[0]), rng.uniform(lo[1], hi[1]), rng.uniform(0.70, 1.10)]
            tris.append(sphere_mesh(c, rng.uniform(0.05, 0.2)))
        p["tri"] = np.concatenate(tris).astype(np.float32) if tris else np.zeros((0, 12), np.float32)
        p["ncand"] = cand_per_template
        parts.append(p)
    return _pack(parts, name=f"meshes T={n_templates}x{cand_per_template}")


def random_poses(batch: SceneBatch, seed: int, spread: float = 0.6) -> np.ndarray:
    """Arbitrary object poses (float32 [P,4]: x, y, z, yaw) for exercising the
    collision check on its own: xy uniform in [-spread, spread]^2 around the
    support, z = support + U(0, 0.3), yaw U(0, 2pi)."""
    rng = np.random.default_rng(seed)
    n = batch.n_poses()
    p = np.empty((n, 4), dtype=np.float64)
    p[:, 0] = rng.uniform(-spread, spread, n)
    p[:, 1] = rng.uniform(-spread, spread, n)
    zs = np.repeat(batch.tmpl_support_z.astype(np.float64), np.diff(batch.tmpl_pose_off()))
    p[:, 2] = zs + rng.uniform(0.0, 0.3, n)
    p[:, 3] = rng.uniform(0.0, 2 * math.pi, n)
    return p.astype(np.float32)


def topdown_targets(seed: int, n: int, box=((0.0, 1.2), (-0.4, 0.4), (0.02, 0.5))) -> np.ndarray:
    """Top-down grasp targets in the robot base frame (float32 [n,12]: R row-major, p).

    Positions are uniform in `box` (metres, base frame; the default covers a
    1.2 x 0.8 m table whose near edge holds the robot, heights from a resting
    object's top up to a stacked one). The tool z axis points down, the tool x
    axis is at a uniform yaw psi: columns x = (cos, sin, 0), y = (sin, -cos, 0),
    z = (0, 0, -1)."""
    rng = np.random.default_rng(seed)
    t = np.zeros((n, 12), dtype=np.float64)
    psi = rng.uniform(0.0, 2 * math.pi, n)
    c, s = np.cos(psi), np.sin(psi)
    t[:, 0], t[:, 1], t[:, 2] = c, s, 0.0
    t[:, 3], t[:, 4], t[:, 5] = s, -c, 0.0
    t[:, 6], t[:, 7], t[:, 8] = 0.0, 0.0, -1.0
    for i, (lo, hi) in enumerate(box):
        t[:, 9 + i] = rng.uniform(lo, hi, n)
    return t.astype(np.float32)


def arm_arrays():
    """(d, a, alpha, qmin, qmax) float32 arrays of the 7-DoF arm."""
    f = lambda v: np.array(v, dtype=np.float32)
    return f(ARM_D), f(ARM_A), f(ARM_ALPHA), f([-ARM_QLIM] * 7), f([ARM_QLIM] * 7)
