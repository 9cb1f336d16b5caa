"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the value: a closed form, a library routine written
by someone else (numpy's Philox4x64, scipy's rotations, torch's bfloat16
conversion, numpy.linalg), an invariance, or brute force on hand-made cases.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy import stats

import oracle
import synth
from oracle import mlp
from scenes import tiny_batch

# --------------------------------------------------------------------------- Philox


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((123, 456), (7, 8, 9, 10)),
                                     ((2**64 - 1, 2**63), (2**64 - 2, 5, 6, 7)), ((1, 2), (2**64 - 1, 0, 0, 0))])
def test_philox4x64_matches_numpy(key, ctr):
    """numpy.random.Philox is Philox4x64-10 and encrypts counter+1 for its first
    block. The oracle's 4x64 instance shares the round, permutation and key
    schedule code with the 4x32 instance the sampler uses."""
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    raw = [int(x) for x in g.random_raw(8)]
    c = list(ctr)
    outs = []
    for _ in range(2):
        c[0] = (c[0] + 1) % 2**64
        if c[0] == 0:
            c[1] = (c[1] + 1) % 2**64
        outs += [int(x) for x in oracle.philox4x64(c, key)]
    assert raw == outs


def _kat_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            rows.append([int(x, 16) for x in line])
    return rows


def test_philox4x32_known_answers():
    """The published Philox4x32-10 known-answer vectors (tests/golden, from the
    Random123 distribution of Salmon et al., SC'11): they fix the multipliers,
    the Weyl key increments and the round count that only statistics covered."""
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        assert [int(x) for x in oracle.philox4x32(r[0:4], r[4:6])] == r[6:10]


def test_philox4x32_statistics():
    """Uniformity (chi^2 on the top byte of every word), full avalanche on a
    one-bit counter change and on a one-bit key change."""
    n = 20000
    words = np.array([oracle.philox4x32([i, 0, 0, 0], [17, 0]) for i in range(n)], dtype=np.uint32)
    top = (words >> 24).ravel()
    chi2, p = stats.chisquare(np.bincount(top, minlength=256))
    assert p > 1e-4, p
    rng = np.random.default_rng(5)
    flips = []
    for _ in range(400):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        a = oracle.philox4x32(ctr, key)
        c2 = ctr.copy(); c2[rng.integers(4)] ^= np.uint32(1 << int(rng.integers(32)))
        k2 = key.copy(); k2[rng.integers(2)] ^= np.uint32(1 << int(rng.integers(32)))
        for b in (oracle.philox4x32(c2, key), oracle.philox4x32(ctr, k2)):
            flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)) / 128.0)
    assert abs(np.mean(flips) - 0.5) < 0.01
    assert min(flips) > 0.25


def test_uniform_is_top_24_bits():
    """u = (x >> 8) 2^-24: a multiple of 2^-24 in [0, 1), same bits as the word."""
    seed = 0x123456789ABCDEF
    w = oracle.philox4x32([3, 1, 2, 5], [seed & 0xFFFFFFFF, seed >> 32])
    u = oracle.uniform4(seed, 3, 1, 2, 5)
    assert np.all(u * 2**24 == (w >> 8).astype(np.float64))
    assert np.all((u >= 0) & (u < 1))


# --------------------------------------------------------------------------- point in polygon

SQUARE = [(0, 0), (1, 0), (1, 1), (0, 1)]
L_SHAPE = [(0, 0), (2, 0), (2, 1), (1, 1), (1, 2), (0, 2)]


@pytest.mark.parametrize("poly", [SQUARE, SQUARE[::-1]])
@pytest.mark.parametrize("p,inside,dist", [((0.5, 0.5), True, 0.5), ((1.5, 0.5), False, 0.5), ((1.0, 0.5), True, 0.0),
                                           ((0.0, 0.0), True, 0.0), ((-1, -1), False, math.sqrt(2)),
                                           ((-0.5, 0.0), False, 0.5), ((0.9, 0.2), True, 0.1)])
def test_pip_square(poly, p, inside, dist):
    got_in, got_d = oracle.point_in_polygon(poly, p)
    assert got_in == inside
    assert got_d == pytest.approx(dist, abs=1e-12)


@pytest.mark.parametrize("poly", [L_SHAPE, L_SHAPE[::-1]])
@pytest.mark.parametrize("p,inside,dist", [((1.5, 1.5), False, 0.5), ((0.5, 1.5), True, 0.5), ((1.5, 0.5), True, 0.5),
                                           ((1.2, 1.1), False, 0.1), ((0.5, 1.0), True, 0.5), ((3.0, 1.0), False, 1.0),
                                           ((1.0, 1.5), True, 0.0)])
def test_pip_concave(poly, p, inside, dist):
    got_in, got_d = oracle.point_in_polygon(poly, p)
    assert got_in == inside
    assert got_d == pytest.approx(dist, abs=1e-12)


def test_pip_random_convex_against_halfplanes():
    """For a convex CCW polygon, inside <=> left of (or on) every edge line;
    an independent test from the crossing-number walk."""
    rng = np.random.default_rng(0)
    poly = synth.convex_polygon(rng, 7, 1.3).astype(np.float64)
    for _ in range(2000):
        p = rng.uniform(-1, 1, 2)
        e = np.roll(poly, -1, axis=0) - poly
        cross = e[:, 0] * (p[1] - poly[:, 1]) - e[:, 1] * (p[0] - poly[:, 0])
        got, d = oracle.point_in_polygon(poly, p)
        assert got == bool(np.all(cross >= 0))
        if got:  # distance to the boundary of a convex polygon = min distance to edge lines
            assert d == pytest.approx(np.min(cross / np.hypot(e[:, 0], e[:, 1])), abs=1e-12)


# --------------------------------------------------------------------------- distances


def test_sphere_sphere_closed_form():
    """Two spheres of radius r at centre distance D: d = D - 2r; collide iff D < 2r."""
    r = 0.03
    for D in np.linspace(0.0, 0.2, 41):
        a = [0.1, -0.2, 0.7, r]
        b = [0.1 + D * 0.6, -0.2 + D * 0.8, 0.7, r]
        d = oracle.sphere_sphere(a, b)
        assert d == pytest.approx(D - 2 * r, abs=1e-15)
        assert oracle.sphere_sphere(b, a) == d
        if abs(D - 2 * r) > 1e-12:  # exact contact is a band case
            assert (d < 0) == (D < 2 * r)


BOX_C, BOX_H = (1.0, 2.0, 3.0), (0.5, 1.0, 2.0)


def _box(centre=BOX_C, quat=(0, 0, 0, 1), half=BOX_H):
    return np.array([*centre, 0, *quat, *half, 0], dtype=np.float32)


@pytest.mark.parametrize("p,expect", [
    ((1.8, 2.0, 3.0), 0.3),                                        # face
    ((1.8, 3.4, 3.0), 0.5),                                        # edge (0.3, 0.4)
    ((1.5 + 0.1, 3.0 + 0.2, 5.0 + 0.2), math.sqrt(0.09)),          # corner (0.1, 0.2, 0.2)
    ((1.2, 2.0, 3.0), -0.3),                                       # interior: nearest face 0.3 away
    ((1.0, 2.0, 3.0), -0.5),                                       # centre
    ((1.0, 2.9, 3.0), -0.1),                                       # interior near the y face
])
def test_sphere_obb_closed_forms(p, expect):
    r = 0.05
    assert oracle.sphere_obb([*p, r], _box()) == pytest.approx(expect - r, abs=1e-6)


def test_sphere_obb_rotation_invariance_and_quat_scale():
    """Rotating box and sphere together about the box centre leaves d unchanged;
    the quaternion is normalised (a scaled quaternion gives the same box)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        R = Rotation.random(random_state=rng)
        q = R.as_quat()  # (x, y, z, w)
        local = rng.uniform(-3, 3, 3)
        r = rng.uniform(0.0, 0.1)
        d_axis = oracle.sphere_obb([*(np.array(BOX_C) + local), r], _box())
        world = np.array(BOX_C) + R.apply(local)
        box = _box(quat=tuple(q))
        d_rot = oracle.sphere_obb([*world, r], box)
        assert d_rot == pytest.approx(d_axis, abs=2e-6)  # float32 quaternion storage
        box2 = _box(quat=tuple(2.5 * q))
        assert oracle.sphere_obb([*world, r], box2) == pytest.approx(d_rot, abs=2e-6)


def test_sphere_world_yaw():
    """Yaw pi/2 maps the local (x, y) to (-y, x); z is shifted, r kept."""
    w = oracle.sphere_world([0.1, 0.2, 0.3, 0.04], [1.0, 2.0, 3.0, math.pi / 2])
    assert np.allclose(w, [1.0 - 0.2, 2.0 + 0.1, 3.3, 0.04], atol=1e-7)


# --------------------------------------------------------------------------- collision on hand-made scenes


def test_collide_brute_force_tiny():
    """(Radii are stored as float32, hence 1e-7.) Three one/two-sphere objects at hand-placed poses; every pair distance
    computed by hand: objects 0-1: centres 0.5 apart, radii 0.1+0.1 -> 0.3;
    0-2: centres 0.25 apart -> 0.05 (second sphere of object 2 at 0.25+0.1
    in x); 1-2: far."""
    b = tiny_batch([[(0, 0, 0, 0.1)], [(0, 0, 0, 0.1)], [(0, 0, 0, 0.1), (0.1, 0, 0, 0.1)]])
    poses = np.array([[0, 0, 0, 0], [0.5, 0, 0, 0], [0, 0.45, 0, 0]], np.float64)
    col, md, band = oracle.collide(b, poses)
    # 0-2: sphere (0,0.45) vs (0,0): 0.45-0.2 = 0.25; sphere (0.1,0.45) vs (0,0): sqrt(0.01+0.2025)-0.2
    d02 = min(0.25, math.sqrt(0.01 + 0.2025) - 0.2)
    d12 = min(math.hypot(0.5, 0.45) - 0.2, math.hypot(0.4, 0.45) - 0.2)
    assert md[0] == pytest.approx(min(0.3, d02, d12), abs=1e-7)
    assert col[0] == 0
    # first_new = 2: only pairs with object 2
    _, md2, _ = oracle.collide(b, poses, first_new=2)
    assert md2[0] == pytest.approx(min(d02, d12), abs=1e-7)
    # first_new = 3: nothing new -> +FLT_MAX
    _, md3, _ = oracle.collide(b, poses, first_new=3)
    assert md3[0] == pytest.approx(np.finfo(np.float32).max)
    # yaw pi of object 2 moves its second sphere to x = -0.1
    poses[2, 3] = math.pi
    _, md4, _ = oracle.collide(b, poses, first_new=2)
    assert md4[0] == pytest.approx(min(0.25, math.hypot(0.5, 0.45) - 0.2, math.hypot(0.6, 0.45) - 0.2), abs=1e-7)


def test_collide_touching_is_free_and_overlap_collides():
    b = tiny_batch([[(0, 0, 0, 0.125)], [(0, 0, 0, 0.125)]])
    col, md, band = oracle.collide(b, np.array([[0, 0, 0, 0], [0.25, 0, 0, 0]], np.float64))
    assert md[0] == 0.0 and col[0] == 0 and band[0] == 1
    col, md, band = oracle.collide(b, np.array([[0, 0, 0, 0], [0.2, 0, 0, 0]], np.float64))
    assert md[0] == pytest.approx(-0.05) and col[0] == 1 and band[0] == 0


def test_collide_world_only_and_intra_object_ignored():
    """Spheres of one object overlapping each other never count; a sphere
    inside a world box does."""
    b = tiny_batch([[(0, 0, 0, 0.1), (0.05, 0, 0, 0.1)]], obbs=[[3, 0, 0, 0, 0, 0, 0, 1, 0.5, 0.5, 0.5, 0]])
    col, md, _ = oracle.collide(b, np.array([[0, 0, 0, 0]], np.float64))
    assert md[0] == pytest.approx(2.5 - 0.05 - 0.1, abs=1e-7) and col[0] == 0
    col, md, _ = oracle.collide(b, np.array([[2.9, 0, 0, 0]], np.float64))
    assert md[0] == pytest.approx(-(0.5 - 0.05) - 0.1, abs=1e-6) and col[0] == 1


def _shelf_small(n_cand=6, n_obj=6, n_sph=5, n_obb=4, seed=11):
    return synth.shelf(seed=seed, n_cand=n_cand, n_obj=n_obj, n_sph=n_sph, n_obb=n_obb)


def test_collide_rigid_motion_invariance():
    """A global yaw psi and translation applied to every object pose and world
    box leaves every signed distance unchanged (up to float32 input storage)."""
    b = _shelf_small()
    poses = synth.random_poses(b, seed=3, spread=0.5).astype(np.float64)
    col, md, _ = oracle.collide(b, poses)
    psi, t = 0.7, np.array([0.3, -0.2, 0.1])
    c, s = math.cos(psi), math.sin(psi)
    p2 = poses.copy()
    p2[:, 0] = c * poses[:, 0] - s * poses[:, 1] + t[0]
    p2[:, 1] = s * poses[:, 0] + c * poses[:, 1] + t[1]
    p2[:, 2] = poses[:, 2] + t[2]
    p2[:, 3] = poses[:, 3] + psi
    obb = b.obb.astype(np.float64).copy()
    obb[:, 0] = c * b.obb[:, 0] - s * b.obb[:, 1] + t[0]
    obb[:, 1] = s * b.obb[:, 0] + c * b.obb[:, 1] + t[1]
    obb[:, 2] = b.obb[:, 2] + t[2]
    q = (Rotation.from_euler("z", psi) * Rotation.from_quat(b.obb[:, 4:8].astype(np.float64))).as_quat()
    obb[:, 4:8] = q
    import dataclasses
    b2 = dataclasses.replace(b, obb=obb.astype(np.float32))
    col2, md2, _ = oracle.collide(b2, p2)
    assert np.allclose(md, md2, atol=2e-6)
    assert np.array_equal(col[np.abs(md) > 1e-5], col2[np.abs(md) > 1e-5])


def test_collide_object_relabelling_invariance():
    """Whole-scene minimum distance does not depend on the object order."""
    b = _shelf_small(n_obb=0)
    poses = synth.random_poses(b, seed=4, spread=0.4).astype(np.float64)
    _, md, _ = oracle.collide(b, poses)
    n_obj = b.n_obj_of(0)
    perm = np.random.default_rng(0).permutation(n_obj)
    spheres = [b.sph_local[b.obj_sph_off[o]:b.obj_sph_off[o + 1]] for o in range(n_obj)]
    b2 = tiny_batch([spheres[k].tolist() for k in perm], n_cand=b.n_cand)
    p2 = poses.reshape(b.n_cand, n_obj, 4)[:, perm].reshape(-1, 4)
    _, md2, _ = oracle.collide(b2, p2)
    assert np.allclose(md, md2, atol=1e-12)


# --------------------------------------------------------------------------- sampler


def test_free_samples_uniform_on_table():
    """Free objects on the 1.2 x 0.8 table: x, y, yaw uniform (KS); z = table + Hz."""
    b = synth.tabletop(seed=0, n_cand=4000)
    P, ok, band = oracle.sample_poses(b, seed=9)
    assert ok.all()
    P = P.reshape(4000, 8, 4)
    for k in range(8):
        assert stats.kstest(P[:, k, 0], stats.uniform(-0.6, 1.2).cdf).pvalue > 1e-4
        assert stats.kstest(P[:, k, 1], stats.uniform(-0.4, 0.8).cdf).pvalue > 1e-4
        assert stats.kstest(P[:, k, 3], stats.uniform(0, 2 * math.pi).cdf).pvalue > 1e-4
        assert np.allclose(P[:, k, 2], 0.75 + b.obj_half[k, 2], atol=1e-7)
    # the same counters give the same poses; another retry index gives others
    P2, _, _ = oracle.sample_poses(b, seed=9)
    assert np.array_equal(P.reshape(-1, 4), P2)
    P3, _, _ = oracle.sample_poses(b, seed=9, retry=1)
    assert not np.any(P3[:, 0] == P.reshape(-1, 4)[:, 0])


def test_convex_support_samples_inside_and_uniform():
    """Accepted xy lie in the polygon (half-plane test), and the fraction on
    each side of a line through the polygon matches the area fraction."""
    rng = np.random.default_rng(4)
    poly = synth.convex_polygon(rng, 6, 1.0)
    b = tiny_batch([[(0, 0, 0, 0.02)]], poly=poly, n_cand=6000)
    P, ok, band = oracle.sample_poses(b, seed=2)
    assert ok.mean() > 0.999
    xy = P[ok.astype(bool), :2]
    e = np.roll(poly, -1, axis=0) - poly
    cross = e[None, :, 0] * (xy[:, None, 1] - poly[None, :, 1]) - e[None, :, 1] * (xy[:, None, 0] - poly[None, :, 0])
    assert np.all(cross >= -1e-12)
    # area left of x = 0 by shoelace on the clipped polygon, via dense grid estimate
    gx, gy = np.meshgrid(np.linspace(-1.5, 1.5, 1201), np.linspace(-1.5, 1.5, 1201))
    g = np.stack([gx.ravel(), gy.ravel()], 1)
    gc = e[None, :, 0] * (g[:, None, 1] - poly[None, :, 1]) - e[None, :, 1] * (g[:, None, 0] - poly[None, :, 0])
    inside = np.all(gc >= 0, axis=1)
    frac = np.mean(g[inside, 0] < 0)
    n = len(xy)
    assert abs(np.mean(xy[:, 0] < 0) - frac) < 4 * math.sqrt(frac * (1 - frac) / n) + 0.005


def test_erosion_ratio_on_support():
    """ratio_on_support = 1 keeps the pivot at least min(Hx, Hy) inside the table edge."""
    b = synth.tabletop(seed=0, n_cand=500)
    b.obj_rel_param[:, 2] = 1.0
    P, ok, _ = oracle.sample_poses(b, seed=3)
    P = P.reshape(500, 8, 4)
    for k in range(8):
        e = min(b.obj_half[k, 0], b.obj_half[k, 1])
        sel = ok.astype(bool)
        assert np.all(np.abs(P[sel, k, 0]) <= 0.6 - e + 1e-9)
        assert np.all(np.abs(P[sel, k, 1]) <= 0.4 - e + 1e-9)


def test_on_top_and_next_to_relations():
    """On-top: bottom of the child = top of the parent (exact), pivot inside the
    parent's top face in the parent frame, uniform there. Next-to: centre
    distance in [rho_a + rho_t + 0.05, rho_a + rho_t + 0.2], on the support."""
    b = synth.shelf(seed=1, n_cand=3000, n_obj=12, n_sph=4, n_obb=0)
    P, ok, band = oracle.sample_poses(b, seed=5)
    P = P.reshape(b.n_cand, 12, 4)
    kinds, refs = b.obj_rel & 0xF, b.obj_rel >> 8
    assert (kinds == synth.REL_ON_TOP).sum() == 3 and (kinds == synth.REL_NEXT_TO).sum() == 3
    H = b.obj_half.astype(np.float64)
    for k in range(12):
        p = refs[k]
        if kinds[k] == synth.REL_ON_TOP:
            assert np.allclose(P[:, k, 2] - H[k, 2], P[:, p, 2] + H[p, 2], atol=1e-12)
            d = P[:, k, :2] - P[:, p, :2]
            c, s = np.cos(P[:, p, 3]), np.sin(P[:, p, 3])
            xl, yl = c * d[:, 0] + s * d[:, 1], -s * d[:, 0] + c * d[:, 1]
            assert np.all(np.abs(xl) <= H[p, 0] + 1e-12) and np.all(np.abs(yl) <= H[p, 1] + 1e-12)
            assert stats.kstest(xl / H[p, 0], stats.uniform(-1, 2).cdf).pvalue > 1e-4
        elif kinds[k] == synth.REL_NEXT_TO:
            dist = np.hypot(P[:, k, 0] - P[:, p, 0], P[:, k, 1] - P[:, p, 1])
            lo, hi = H[p, 3] + H[k, 3] + 0.05, H[p, 3] + H[k, 3] + 0.2
            sel = ok.astype(bool)
            assert np.all(dist[sel] >= lo - 1e-12) and np.all(dist[sel] <= hi + 1e-12)
            assert np.all(np.abs(P[sel, k, 0]) <= 0.6) and np.all(np.abs(P[sel, k, 1]) <= 0.4)
            assert np.allclose(P[:, k, 2], 0.75 + H[k, 2])


# --------------------------------------------------------------------------- generation


def test_generate_valid_scenes_are_collision_free():
    """Every scene the loop marks valid passes the whole-scene check (all pairs)."""
    b = synth.tabletop(seed=0, n_cand=256)
    P, valid, band, tries = oracle.generate(b, seed=1)
    assert valid.mean() > 0.5
    sel = np.nonzero(valid)[0]
    col, md, cb = oracle.collide(b, P, active=sel.astype(np.int32))
    assert np.all(md >= -1e-12)
    assert np.all(tries[valid.astype(bool)] >= 8) and np.all(tries <= 8 * 11)


def test_generate_without_retries_equals_whole_scene_check():
    """With no retries every object keeps its retry-0 sample, so a scene is valid
    exactly when the retry-0 samples are all accepted and the whole scene is
    collision-free: the incremental per-object checks cover every pair once."""
    b = synth.tabletop(seed=0, n_cand=512)
    P, valid, band, _ = oracle.generate(b, seed=2, max_retries=0)
    Ps, ok, sband = oracle.sample_poses(b, seed=2)
    col, md, cband = oracle.collide(b, Ps)
    whole = ok.astype(bool) & (md >= 0)
    keep = ~(band.astype(bool) | sband.astype(bool) | cband.astype(bool))
    assert np.array_equal(valid.astype(bool)[keep], whole[keep])
    assert whole.sum() > 0


# --------------------------------------------------------------------------- kinematics

ARM = oracle.make_arm(*synth.arm_arrays())


def _dh_scipy(q, d=synth.ARM_D, a=synth.ARM_A, alpha=synth.ARM_ALPHA):
    T = np.eye(4)
    for i in range(7):
        Rz = np.eye(4); Rz[:3, :3] = Rotation.from_euler("z", q[i]).as_matrix()
        Tz = np.eye(4); Tz[2, 3] = float(np.float32(d[i]))
        Tx = np.eye(4); Tx[0, 3] = float(np.float32(a[i]))
        Rx = np.eye(4); Rx[:3, :3] = Rotation.from_euler("x", float(np.float32(alpha[i]))).as_matrix()
        T = T @ Rz @ Tz @ Tx @ Rx
    return T


# The workloads' arm has twists 0 and +-pi/2 only, whose cosines or sines
# vanish; these two make every term of the DH product count.
OTHER_ARMS = {
    "iiwa-like": ([0.34, 0.0, 0.4, 0.0, 0.4, 0.0, 0.126], [0.0] * 7,
                  [-math.pi / 2, math.pi / 2, math.pi / 2, -math.pi / 2, -math.pi / 2, math.pi / 2, 0.0]),
    "general": (list(synth.ARM_D), list(synth.ARM_A), [0.3, -1.2, 0.9, 1.4, -0.7, 1.1, 0.5]),
}


@pytest.mark.parametrize("name", sorted(OTHER_ARMS))
def test_fk_and_jacobian_on_other_arms(name):
    d, a, alpha = OTHER_ARMS[name]
    f = lambda v: np.array(v, np.float32)
    arm = oracle.make_arm(f(d), f(a), f(alpha), f([-2.8] * 7), f([2.8] * 7))
    rng = np.random.default_rng(12)
    h = 1e-6
    for q in [np.zeros(7)] + [rng.uniform(-2.8, 2.8, 7) for _ in range(10)]:
        assert np.allclose(oracle.fk_frames(arm, q)[7], _dh_scipy(q, d, a, alpha), atol=1e-7)
        J = oracle.jacobian(arm, q)
        for i in range(7):
            dq = np.zeros(7); dq[i] = h
            Fp, Fm = oracle.fk_frames(arm, q + dq)[7], oracle.fk_frames(arm, q - dq)[7]
            assert np.allclose(J[:3, i], (Fp[:3, 3] - Fm[:3, 3]) / (2 * h), atol=1e-7)
            assert np.allclose(J[3:, i], Rotation.from_matrix(Fp[:3, :3] @ Fm[:3, :3].T).as_rotvec() / (2 * h),
                               atol=1e-7)


def test_fk_matches_scipy_dh_chain():
    rng = np.random.default_rng(2)
    for q in [np.zeros(7)] + [rng.uniform(-2.8, 2.8, 7) for _ in range(20)]:
        F = oracle.fk_frames(ARM, q)
        assert np.allclose(F[7], _dh_scipy(q), atol=1e-7)  # float32 DH parameters
    # hand product at q = 0: Tz(d1); Rx(-pi/2); Tz(d3) along world +y; Rx(pi/2) -> R = I;
    # Tx(a4); Rx(pi/2); Tz(d5) along world -y; Tx(a5); Rx(-pi/2) -> I; Rx(pi/2);
    # Tz(d7) along -y; Tx(a7); Rx(pi/2): p = (a4 + a5 + a7, d3 - d5 - d7, d1), R = Rx(pi)
    F0 = oracle.fk_frames(ARM, np.zeros(7))[7]
    assert np.allclose(F0[:3, 3], [0.088, 0.316 - 0.384 - 0.107, 0.333], atol=1e-7)
    assert np.allclose(F0[:3, :3], np.diag([1.0, -1.0, -1.0]), atol=1e-6)


def test_jacobian_matches_finite_differences():
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(10):
        q = rng.uniform(-2.5, 2.5, 7)
        J = oracle.jacobian(ARM, q)
        for i in range(7):
            dq = np.zeros(7); dq[i] = h
            Fp, Fm = oracle.fk_frames(ARM, q + dq)[7], oracle.fk_frames(ARM, q - dq)[7]
            v = (Fp[:3, 3] - Fm[:3, 3]) / (2 * h)
            w = Rotation.from_matrix(Fp[:3, :3] @ Fm[:3, :3].T).as_rotvec() / (2 * h)
            assert np.allclose(J[:3, i], v, atol=1e-7)
            assert np.allclose(J[3:, i], w, atol=1e-7)


def test_orientation_error_and_angle_closed_forms():
    """R* = Rot(a, delta) R  =>  1/2 sum r_k x r*_k = sin(delta) a and the
    rotation angle of R^T R* is delta; the position part is p* - p."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        q = rng.uniform(-2.5, 2.5, 7)
        T = oracle.fk_frames(ARM, q)[7]
        a = rng.normal(size=3); a /= np.linalg.norm(a)
        delta = rng.uniform(0.0, 3.0)
        Rs = Rotation.from_rotvec(delta * a).as_matrix() @ T[:3, :3]
        dp = rng.normal(size=3) * 0.1
        tgt = np.concatenate([Rs.ravel(), T[:3, 3] + dp])
        e = oracle.ik_error(ARM, q, tgt)
        assert np.allclose(e[:3], dp, atol=1e-12)
        assert np.allclose(e[3:], math.sin(delta) * a, atol=1e-12)
        pe, re = oracle.pose_error(ARM, q, tgt)
        assert pe == pytest.approx(np.linalg.norm(dp), abs=1e-12)
        assert re == pytest.approx(delta, abs=1e-9)


def test_dls_step_push_through_identity():
    """J^T (J J^T + l^2 I)^-1 e == (J^T J + l^2 I)^-1 J^T e (numpy.linalg.solve)."""
    rng = np.random.default_rng(5)
    lam = 0.05
    for _ in range(20):
        q = rng.uniform(-1.5, 1.5, 7)
        T = oracle.fk_frames(ARM, q)[7]
        tgt = np.concatenate([(Rotation.from_rotvec(rng.normal(size=3) * 0.05).as_matrix() @ T[:3, :3]).ravel(),
                              T[:3, 3] + rng.normal(size=3) * 0.02])
        J = oracle.jacobian(ARM, q)
        e = oracle.ik_error(ARM, q, tgt)
        dq = np.linalg.solve(J.T @ J + lam**2 * np.eye(7), J.T @ e)
        assert np.all(np.abs(q + dq) < 2.8)
        assert np.allclose(oracle.dls_step(ARM, lam, q, tgt) - q, dq, atol=1e-10)


def test_ik_reaches_fk_targets_and_never_beyond_reach():
    rng = np.random.default_rng(6)
    P = oracle.ik_params(seeds=8, iters=100)
    qs = rng.uniform(-2.5, 2.5, (40, 7))
    tg = np.array([np.concatenate([oracle.fk_frames(ARM, q)[7][:3, :3].ravel(), oracle.fk_frames(ARM, q)[7][:3, 3]])
                   for q in qs], np.float32)
    reach, qo, err, _ = oracle.ik_reach(ARM, P, tg)
    assert reach.mean() >= 0.8
    for i in np.nonzero(reach)[0]:
        pe, re = oracle.pose_error(ARM, qo[i], tg[i].astype(np.float64))
        assert pe <= 5e-3 and re <= 0.05
        assert np.all(np.abs(qo[i]) <= 2.8)
    # the tool can never be farther from the base origin than sum(|d_i| + |a_i|)
    bound = sum(abs(x) for x in synth.ARM_D) + sum(abs(x) for x in synth.ARM_A)
    far = synth.topdown_targets(7, 30, box=((1.45, 2.0), (-0.5, 0.5), (-0.3, 0.3)))
    assert np.all(np.linalg.norm(far[:, 9:], axis=1) > bound)
    reach, _, _, _ = oracle.ik_reach(ARM, P, far)
    assert reach.sum() == 0


@pytest.mark.parametrize("name", ["workload"] + sorted(OTHER_ARMS))
def test_reach_bound_of_the_generation_rounds(name):
    """The rounds reject a try whose grasp target lies farther than
    |a_0| + sum_{i>0} sqrt(a_i^2 + d_i^2) + tol_pos + 1e-4 from (0, 0, d_0),
    or whose wrist point lies beyond the wrist bound: the tool never leaves
    that ball (every link adds a_i x_i + d_i z_i with x_i perpendicular to
    z_i), nor the wrist its ball, and targets just beyond either bound are
    unreachable and unbanded for the exact IK."""
    if name == "workload":
        d, a, alpha = synth.ARM_D, synth.ARM_A, synth.ARM_ALPHA
    else:
        d, a, alpha = OTHER_ARMS[name]
    f = lambda v: np.array(v, np.float32)
    arm = oracle.make_arm(f(d), f(a), f(alpha), f([-2.8] * 7), f([2.8] * 7))
    d32, a32 = f(d).astype(np.float64), f(a).astype(np.float64)
    rmax = abs(a32[0]) + np.sum(np.sqrt(a32[1:] ** 2 + d32[1:] ** 2))
    shoulder = np.array([0.0, 0.0, d32[0]])
    rng = np.random.default_rng(13)
    far_q = max(np.linalg.norm(oracle.fk_frames(arm, q)[7][:3, 3] - shoulder)
                for q in rng.uniform(-2.8, 2.8, (2000, 7)))
    assert far_q <= rmax + 1e-9 and far_q >= 0.9 * rmax  # the ball bounds the tool, not loosely
    tol_pos = 5e-3
    n = 64
    u = rng.normal(size=(n, 3)); u /= np.linalg.norm(u, axis=1, keepdims=True)
    pos = shoulder + u * (rmax + tol_pos + 1e-4 + rng.uniform(0.0, 2e-3, (n, 1)))
    rot = Rotation.random(n, random_state=7).as_matrix().reshape(n, 9)
    tg = np.concatenate([rot, pos], axis=1).astype(np.float32)
    reach, _, _, _, band = oracle.ik_reach(arm, oracle.ik_params(seeds=8, iters=100), tg, with_band=True)
    assert reach.sum() == 0 and band.sum() == 0
    # the wrist bound: frame 6's origin is t - R v with v = (a_6, d_6 sin alpha_6,
    # d_6 cos alpha_6) in the tool frame, within r6 (links 1..5) of the shoulder;
    # a target whose t* - R* v lies beyond r6 + tol_pos + 2 sin(tol_rot / 2) |v|
    # (+ the band's 1e-5 on both tolerances and 1e-4) fails with no band
    al6 = float(np.float32(alpha[6]))
    v = np.array([a32[6], d32[6] * math.sin(al6), d32[6] * math.cos(al6)])
    r6 = abs(a32[0]) + np.sum(np.sqrt(a32[1:6] ** 2 + d32[1:6] ** 2))
    for q in rng.uniform(-2.8, 2.8, (200, 7)):
        F = oracle.fk_frames(arm, q)
        assert np.allclose(F[7][:3, 3] - F[7][:3, :3] @ v, F[6][:3, 3], atol=1e-9)
        assert np.linalg.norm(F[6][:3, 3] - shoulder) <= r6 + 1e-9
    tol_rot = 0.05
    b6 = r6 + tol_pos + 1e-5 + 2 * math.sin((tol_rot + 1e-5) / 2) * np.linalg.norm(v) + 1e-4
    u = rng.normal(size=(n, 3)); u /= np.linalg.norm(u, axis=1, keepdims=True)
    R = Rotation.random(n, random_state=8).as_matrix()
    pw = shoulder + u * (b6 + rng.uniform(0.0, 2e-3, (n, 1)))
    pos = pw + np.einsum("nij,j->ni", R, v)
    tg = np.concatenate([R.reshape(n, 9), pos], axis=1).astype(np.float32)
    reach, _, _, _, band = oracle.ik_reach(arm, oracle.ik_params(seeds=8, iters=100), tg, with_band=True)
    assert reach.sum() == 0 and band.sum() == 0


def _seed_q(seed, target, s, hi=0):
    """Seed s of a target as the documented draw: q_j = qmin + (qmax - qmin) u_j,
    u = (w >> 8) 2^-24 of Philox4x32-10 word j % 4 at counter (target, s, j / 4,
    hi), key = (seed low, seed high); the generator is pinned by its known
    answers above."""
    q = np.zeros(7)
    for b in range(2):
        w = oracle.philox4x32([target, s, b, hi], [seed & 0xFFFFFFFF, seed >> 32])
        for j in range(4):
            if 4 * b + j < 7:
                q[4 * b + j] = -2.8 + 5.6 * float(np.float32(float(int(w[j]) >> 8) * 2.0**-24))
    return q


def test_ik_seed_draw_matches_its_definition():
    for seed, target, s in [(3, 0, 0), (3, 17, 31), (2**40 + 5, 123456, 7)]:
        assert np.allclose(oracle.ik_seed(ARM, seed, target, s), _seed_q(seed, target, s), atol=1e-12)


def _target_of(T):
    return np.concatenate([T[:3, :3].ravel(), T[:3, 3]]).astype(np.float32)


def test_ik_selection_at_zero_iterations():
    """With no step the seeds alone decide. A target made (by scipy's DH chain)
    from seed s's own configuration is reached by the lowest seed whose
    scipy-FK pose meets the tolerances (normally s itself), and its q is
    returned; an unreachable target returns the seed of least scipy-FK
    position error."""
    rng = np.random.default_rng(12)
    P = oracle.ik_params(seeds=8, iters=0, seed=9)
    n = 24
    chosen = rng.integers(0, 8, n)
    seeds = [[_seed_q(9, i, s) for s in range(8)] for i in range(n)]
    tg = np.array([_target_of(_dh_scipy(seeds[i][chosen[i]])) for i in range(n)])
    # the last quarter: moved 0.3 m away, so no seed meets 5 mm
    tg[18:, 9] += 0.3
    reach, qo, err, it = oracle.ik_reach(ARM, P, tg)
    assert np.all(it == 0)
    for i in range(n):
        pes, res = [], []
        for s in range(8):
            T = _dh_scipy(seeds[i][s])
            pes.append(np.linalg.norm(T[:3, 3] - tg[i, 9:].astype(np.float64)))
            Rt = tg[i, :9].astype(np.float64).reshape(3, 3)
            res.append(Rotation.from_matrix(T[:3, :3].T @ Rt).magnitude())
        ok = [s for s in range(8) if pes[s] <= 5e-3 and res[s] <= 0.05]
        if i < 18:
            assert ok and ok[0] <= chosen[i]
            assert reach[i] == 1 and np.allclose(qo[i], seeds[i][ok[0]], atol=1e-12)
        else:
            assert not ok and reach[i] == 0
            assert np.allclose(qo[i], seeds[i][int(np.argmin(pes))], atol=1e-12)
            assert err[i, 0] == pytest.approx(min(pes), abs=1e-6)  # float32 DH lengths in the oracle
    # loose tolerances: several seeds succeed at once; the lowest index wins,
    # not the most accurate one
    P2 = oracle.ik_params(seeds=8, iters=0, seed=9, tol_pos=0.7, tol_rot=1.5)
    reach2, qo2, _, _ = oracle.ik_reach(ARM, P2, tg)
    informative = 0
    for i in range(n):
        pes, oks = [], []
        for s in range(8):
            T = _dh_scipy(seeds[i][s])
            pe = np.linalg.norm(T[:3, 3] - tg[i, 9:].astype(np.float64))
            re = Rotation.from_matrix(T[:3, :3].T @ tg[i, :9].astype(np.float64).reshape(3, 3)).magnitude()
            pes.append(pe)
            if pe <= 0.7 and re <= 1.5:
                oks.append(s)
        assert reach2[i] == (len(oks) > 0)
        if oks:
            assert np.allclose(qo2[i], seeds[i][oks[0]], atol=1e-12)
            informative += len(oks) > 1 and oks[int(np.argmin([pes[s] for s in oks]))] != oks[0]
    assert informative >= 2


def test_ik_band_flag_at_the_position_tolerance():
    """A target whose position lies tol_pos +- 5e-6 from seed 0's tool point
    (same rotation) is banded; at +- 2e-5 it is not, and the decision follows
    the side of the tolerance."""
    P = oracle.ik_params(seeds=4, iters=0, seed=21)
    rows, expect = [], []
    for i, (dr, banded) in enumerate([(-5e-6, 1), (5e-6, 1), (-2e-5, 0), (2e-5, 0)]):
        T = _dh_scipy(_seed_q(21, i, 0))
        u = np.array([0.6, -0.48, 0.64])
        tgt = T[:3, 3] + (5e-3 + dr) * u
        rows.append(np.concatenate([T[:3, :3].ravel(), tgt]).astype(np.float32))
        expect.append((int(dr < 0), banded))
    reach, _, err, _, band = oracle.ik_reach(ARM, P, np.array(rows), with_band=True)
    for i, (r, b) in enumerate(expect):
        assert (reach[i], band[i]) == (r, b), (i, reach[i], band[i], err[i])


def _reach_batch():
    return synth.ragged(seed=31, n_templates=6, cand_per_template=12, obj_range=(2, 7), n_reach=4)


def test_generate_reach_branch_with_tolerances_every_seed_meets():
    """tol_pos = 10 m, tol_rot = pi: IK succeeds at its first check on every
    try, so generation with the arm equals generation without it."""
    b = _reach_batch()
    ikp = oracle.ik_params(tol_pos=10.0, tol_rot=math.pi, iters=5, seeds=4, seed=2)
    p0, v0, b0, t0 = oracle.generate(b, seed=4)
    p1, v1, b1, t1 = oracle.generate(b, seed=4, arm=ARM, ikp=ikp)
    assert 0 < v0.sum() < len(v0)
    assert np.array_equal(v0, v1) and np.array_equal(t0, t1)
    assert np.array_equal(p0, p1, equal_nan=True)
    assert np.all(b1 >= b0)


def test_generate_reach_branch_with_every_grasp_out_of_reach():
    """Base 3 m beyond the support: every grasp lies farther than
    sum |d_i| + |a_i| = 1.393 m, so object 0 (designated, free, no world to
    hit) fails IK on every try, spends exactly max_retries + 1 tries, the
    candidate is invalid and no later object is placed."""
    b = _reach_batch()
    b.tmpl_base[:, 0] -= 3.0
    ikp = oracle.ik_params(iters=3, seeds=4, seed=2)
    for retries in (0, 3):
        poses, v, _, tries = oracle.generate(b, seed=4, max_retries=retries, arm=ARM, ikp=ikp)
        assert v.sum() == 0
        assert np.all(tries == retries + 1)
        offs = oracle.pose_offsets(b)
        t_of = b.cand_template()
        for c in range(b.n_cand):
            n = b.n_obj_of(t_of[c])
            assert np.all(np.isfinite(poses[offs[c]]))
            assert np.all(np.isnan(poses[offs[c] + 1: offs[c] + n]))


def test_grasp_target_frame():
    """Top-down grasp: tool z = -world z, tool x along the object yaw (in the base
    frame), position = top of the object; a base yaw rotates both."""
    base = np.array([-0.6, 0.1, 0.75, 0.3], np.float32)
    pose = np.array([0.2, -0.1, 0.9, 1.1])
    t = oracle.grasp_target(pose, 0.05, base)
    R = t[:9].reshape(3, 3)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) == pytest.approx(1.0)
    assert np.allclose(R[:, 2], [0, 0, -1])
    ang = 1.1 - float(base[3])
    assert np.allclose(R[:, 0], [math.cos(ang), math.sin(ang), 0], atol=1e-7)
    Rb = Rotation.from_euler("z", float(base[3])).as_matrix()
    assert np.allclose(Rb @ t[9:], pose[:3] + [0, 0, 0.05] - base[:3], atol=1e-7)


# --------------------------------------------------------------------------- MLP


def test_bf16_round_matches_torch():
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 65504.0, 3.0e38, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_bce_closed_forms():
    assert mlp.bce_with_logits(0.0, 0.0) == pytest.approx(math.log(2), abs=1e-15)
    assert mlp.bce_with_logits(0.0, 1.0) == pytest.approx(math.log(2), abs=1e-15)
    assert mlp.bce_with_logits(40.0, 1.0) == pytest.approx(math.exp(-40), rel=1e-9)
    assert mlp.bce_with_logits(40.0, 0.0) == pytest.approx(40.0, rel=1e-12)
    z = np.linspace(-5, 5, 11)
    ref = -(np.log(1 / (1 + np.exp(-z))))
    assert np.allclose(mlp.bce_with_logits(z, 1.0), ref, atol=1e-12)


def test_silu_grad_finite_difference():
    a = np.linspace(-6, 6, 101)
    h = 1e-6
    assert np.allclose(mlp.silu_grad(a), (mlp.silu(a + h) - mlp.silu(a - h)) / (2 * h), atol=1e-8)


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    P = mlp.init_params(rng, mu=rng.normal(size=9) * 0.1, sigma=rng.uniform(0.5, 2, 9))
    tg = synth.topdown_targets(3, 6)
    y = rng.integers(0, 2, 6).astype(np.float64)
    L, dW, db = mlp.backward(P, tg, y, bf16=False)
    h = 1e-6
    for l in range(4):
        for _ in range(6):
            i, j = rng.integers(P.W[l].shape[0]), rng.integers(P.W[l].shape[1])
            P.W[l][i, j] += h; Lp = mlp.loss(P, tg, y, bf16=False)
            P.W[l][i, j] -= 2 * h; Lm = mlp.loss(P, tg, y, bf16=False)
            P.W[l][i, j] += h
            assert dW[l][i, j] == pytest.approx((Lp - Lm) / (2 * h), abs=1e-8)
        i = rng.integers(P.b[l].shape[0])
        P.b[l][i] += h; Lp = mlp.loss(P, tg, y, bf16=False)
        P.b[l][i] -= 2 * h; Lm = mlp.loss(P, tg, y, bf16=False)
        P.b[l][i] += h
        assert db[l][i] == pytest.approx((Lp - Lm) / (2 * h), abs=1e-8)


def test_mlp_bf16_close_to_exact():
    """The bf16 rounding points move the loss by O(2^-8) relative, no more."""
    rng = np.random.default_rng(2)
    P = mlp.init_params(rng)
    tg = synth.topdown_targets(4, 64)
    y = rng.integers(0, 2, 64).astype(np.float64)
    assert mlp.loss(P, tg, y, bf16=True) == pytest.approx(mlp.loss(P, tg, y, bf16=False), rel=2e-2)


def test_adam_first_step_closed_form():
    """From zero moments the bias-corrected first step is -lr g / (|g| + eps)."""
    g = np.array([1e-3, -2.0, 0.5, 0.0])
    w0 = np.array([1.0, 2.0, 3.0, 4.0])
    w1, m, v = mlp.adam_step(w0, g, np.zeros(4), np.zeros(4), 1)
    assert np.allclose(w1 - w0, -1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


# --------------------------------------------------------------------------- 4D reachability map

from oracle import rmap  # noqa: E402

RM_P = (10, 4, 10, 0.0, 1.0, 1.0)  # nz, nc, nxy, z_lo, z_hi, r_max: 0.1 m / 0.5 (cosine) / 0.2 m bins


def _target(R, p):
    return np.concatenate([np.asarray(R, np.float64).reshape(9), p]).astype(np.float32)


def _topdown(p, yaw):
    """Tool z down, tool x at angle yaw in the horizontal plane (rotation matrix by hand)."""
    c, s = math.cos(yaw), math.sin(yaw)
    return _target([[c, s, 0], [s, -c, 0], [0, 0, -1]], p)


def test_rmap_cell_hand_computed():
    """Top-down grasp at p = (0.55, 0, 0.25), tool x along +x: the reference
    direction is the tool x axis, so x* = 0.55, y* = 0, tilt cosine -1: bins
    (iz, ic, ix, iy) = (2, 0, 7, 5) by hand -> ((2*4 + 0)*10 + 7)*10 + 5."""
    assert rmap.cells(RM_P, _topdown([0.55, 0.0, 0.25], 0.0)[None])[0] == 875
    # tool x along +y: the frame turns by 90 deg, the same point lies on y* = -0.55
    # (ix = floor(1.0 * 5) = 5, iy = floor(0.45 * 5) = 2)
    assert rmap.cells(RM_P, _topdown([0.55, 0.0, 0.25], math.pi / 2)[None])[0] == ((2 * 4 + 0) * 10 + 5) * 10 + 2
    # approach tilted 90 deg (horizontal, along +y): a_z = 0 -> tilt bin 2; the
    # reference is a itself: x* = p.y, y* = -p.x
    R = Rotation.from_euler("x", -90, degrees=True).as_matrix()  # maps e_z to +y
    assert np.allclose(R @ [0, 0, 1], [0, 1, 0])
    t = _target(R, [0.1, 0.3, 0.65])
    assert rmap.cells(RM_P, t[None])[0] == ((6 * 4 + 2) * 10 + 6) * 10 + 4


def test_rmap_cell_turn_about_base_z_invariant():
    """Turning the whole target by 90 deg about the base z axis is exact in
    FP32 (a swap and a sign), and the key is built to be invariant under any
    such turn: the same cell, for random orientations."""
    rng = np.random.default_rng(3)
    Rs = Rotation.random(500, random_state=rng).as_matrix()
    ps = rng.uniform([-0.9, -0.9, 0.0], [0.9, 0.9, 1.0], (500, 3))
    t = np.stack([_target(R, p) for R, p in zip(Rs, ps)])
    Q = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], np.float64)
    t2 = np.stack([_target(Q @ R, Q @ p) for R, p in zip(Rs, ps)])
    c1, c2 = rmap.cells(RM_P, t), rmap.cells(RM_P, t2)
    assert (c1 >= 0).sum() > 300
    assert np.array_equal(c1, c2)


def test_rmap_outside_and_degenerate_have_no_cell():
    bad = np.stack([_topdown([0.0, 0.0, 1.2], 0.0), _topdown([1.5, 0.0, 0.5], 0.0), _topdown([0.0, 0.0, -0.01], 0.0),
                    np.zeros(12, np.float32), np.full(12, np.nan, np.float32)])
    assert np.all(rmap.cells(RM_P, bad) == -1)


def test_rmap_counts_and_scores():
    """Counts conserve the in-grid labels; a cell's score is floor(65535 p / n)
    (1 of 3 -> 21845), 65535 without labels, 0 outside the grid; every reachable training target
    passes tau = 1 when no cell holds more than 65535 labels, so tuning for
    recall 1 on the build set gives recall 1."""
    rng = np.random.default_rng(4)
    n = 4000
    t = np.stack([_topdown(p, y) for p, y in zip(rng.uniform([-1.1, -1.1, -0.1], [1.1, 1.1, 1.1], (n, 3)),
                                                 rng.uniform(0, 2 * math.pi, n))])
    y = (rng.uniform(size=n) < 0.4).astype(np.uint8)
    c = rmap.cells(RM_P, t)
    counts = rmap.build(RM_P, t, y)
    assert counts[:, 1].sum() == (c >= 0).sum() and counts[:, 0].sum() == ((c >= 0) & (y == 1)).sum()
    s = rmap.score(RM_P, counts, t)
    assert np.all(s[(c >= 0) & (y == 1)] >= 1) and np.all(s[c < 0] == 0)
    inside = c >= 0
    tau, rec, pr = rmap.tune(s[inside], y[inside], 1.0)
    assert tau >= 1 and rec == 1.0 and pr < 1.0
    one = np.zeros((rmap.n_cells(RM_P), 2), np.uint32)
    one[875] = (1, 3)
    assert rmap.score(RM_P, one, _topdown([0.55, 0.0, 0.25], 0.0)[None])[0] == 21845
    assert rmap.score(RM_P, one, _topdown([0.15, 0.0, 0.25], 0.0)[None])[0] == 65535  # an empty cell


# --------------------------------------------------------------------------- Sec. IV-F relation set

BIG = ((-50, -50), (50, -50), (50, 50), (-50, 50))  # a support no proposal leaves
ONE = [(0.0, 0.0, 0.0, 0.01)]


def _fixed_anchor_samples(rel, relp, dirs, n_cand, anchors=None, n_obj=2, anchor_poses=None, poly=BIG, seed=21):
    """Sample the last object of a tiny template with the earlier objects
    placed at anchor_poses (x, y, z, yaw) in every candidate."""
    b = tiny_batch([ONE] * n_obj, poly=poly, n_cand=n_cand, rel=rel, relp=relp, dirs=dirs, anchors=anchors)
    poses = np.zeros((b.n_poses(), 4))
    for k, p in enumerate(anchor_poses):
        poses[k::n_obj] = p
    p, ok, band = oracle.sample_poses(b, seed=seed, first_obj=n_obj - 1, n_obj=1, poses=poses)
    return p[n_obj - 1::n_obj], ok, band


def test_directional_sector_area_uniform():
    """DIRECTIONAL with v at 40 deg in the anchor's frame (anchor yaw 30 deg),
    theta = 25 deg, radii [0.3, 0.9] m on a support no proposal leaves: every
    point lies in the sector, r^2 is uniform on [0.09, 0.81] and the angle
    uniform on v +- theta (area-uniform over the partial annulus)."""
    th, yaw_a, v = math.radians(25), math.radians(30), math.radians(40)
    rel = [0, synth.REL_DIRECTIONAL | synth.REL_LOCAL]
    relp = [[0.05, 0.2, 0, 0], [0.3, 0.9, 0, th]]
    p, ok, band = _fixed_anchor_samples(rel, relp, [0, v], 4000, anchor_poses=[(1.0, -2.0, 0.0, yaw_a)])
    assert ok.all() and not band.any()
    d = p[:, :2] - [1.0, -2.0]
    r2 = (d ** 2).sum(1)
    ang = np.arctan2(d[:, 1], d[:, 0]) - (v + yaw_a)
    assert r2.min() >= 0.09 - 1e-12 and r2.max() <= 0.81 + 1e-12 and np.abs(ang).max() <= th + 1e-12
    assert stats.kstest(r2, stats.uniform(0.09, 0.72).cdf).pvalue > 1e-3
    assert stats.kstest(ang, stats.uniform(-th, 2 * th).cdf).pvalue > 1e-3


def test_directional_greater_is_cut_at_the_support():
    """max_r = inf ('greater'): the radius range ends at the support box's
    farthest corner from the anchor, and the support decides the rest."""
    sq = ((-1, -1), (1, -1), (1, 1), (-1, 1))
    rel = [0, synth.REL_DIRECTIONAL]
    relp = [[0.05, 0.2, 0, 0], [0.5, math.inf, 0, math.pi]]
    p, ok, band = _fixed_anchor_samples(rel, relp, [0, 0.0], 3000, anchor_poses=[(0.2, 0.0, 0.0, 0.0)], poly=sq)
    d = np.hypot(p[:, 0] - 0.2, p[:, 1])
    assert d.min() >= 0.5 - 1e-12 and d.max() <= math.hypot(1.2, 1.0) + 1e-12
    acc = ok.astype(bool)
    assert acc.mean() > 0.9
    assert np.all(np.abs(p[acc, :2]) <= 1.0 + 1e-12)


def test_middle_triangle_and_segment():
    """MIDDLE of three anchors: every accepted point is inside the triangle and
    the points are uniform over it (the first barycentric coordinate of a
    uniform point has CDF 1 - (1 - x)^2); of two anchors: on the segment,
    with the position along it uniform."""
    A = np.array([[0.0, 0.0], [1.0, 0.2], [0.3, 0.9]])
    rel = [0, 0, 0, synth.REL_MIDDLE]
    anchors = [[], [], [], [0, 1, 2]]
    p, ok, band = _fixed_anchor_samples(rel, None, None, 4000, anchors=anchors, n_obj=4,
                                        anchor_poses=[(*A[0], 0, 0), (*A[1], 0, 0), (*A[2], 0, 0)])
    acc = ok.astype(bool) & ~band.astype(bool)
    assert acc.mean() > 0.95
    T = np.array([A[1] - A[0], A[2] - A[0]]).T
    lam = np.linalg.solve(T, (p[acc, :2] - A[0]).T).T
    l0 = 1 - lam.sum(1)
    assert lam.min() >= -1e-9 and l0.min() >= -1e-9
    assert stats.kstest(l0, lambda x: 1 - (1 - np.clip(x, 0, 1)) ** 2).pvalue > 1e-3
    rel2, anchors2 = [0, 0, synth.REL_MIDDLE], [[], [], [1, 0]]
    q, ok2, _ = _fixed_anchor_samples(rel2, None, None, 3000, anchors=anchors2, n_obj=3,
                                      anchor_poses=[(0.5, 0.5, 0, 0), (-0.5, 0.1, 0, 0)])
    t = (q[:, 0] - (-0.5)) / 1.0
    assert ok2.all()
    assert np.allclose(q[:, 1], 0.1 + t * 0.4, atol=1e-12)
    assert stats.kstest(t, stats.uniform(0, 1).cdf).pvalue > 1e-3


def test_face_to_points_at_the_reference():
    """FACE_TO on a free object: its yaw points from it to the reference."""
    rel = [0, synth.REL_FACE_TO | (0 << 8)]
    p, ok, _ = _fixed_anchor_samples(rel, None, None, 500, anchor_poses=[(0.3, -0.4, 0.0, 1.0)],
                                     poly=((-1, -1), (1, -1), (1, 1), (-1, 1)))
    d = np.array([0.3, -0.4]) - p[:, :2]
    u = np.stack([np.cos(p[:, 3]), np.sin(p[:, 3])], 1)
    assert np.allclose((u * d).sum(1), np.hypot(d[:, 0], d[:, 1]), atol=1e-12)


def test_bad_relations_sample_free():
    """A MIDDLE object with one anchor, or one naming a later object, and a
    DIRECTIONAL one referring forward are sampled as free objects (the same
    draws as a free object)."""
    free, _, _ = _fixed_anchor_samples([0, 0, 0], None, None, 50, n_obj=3, anchor_poses=[(0, 0, 0, 0), (0.5, 0, 0, 0)],
                                       poly=((-1, -1), (1, -1), (1, 1), (-1, 1)))
    for rel, anchors in (([0, 0, synth.REL_MIDDLE], [[], [], [0]]), ([0, 0, synth.REL_MIDDLE], [[], [], [0, 2]]),
                         ([0, 0, synth.REL_DIRECTIONAL | (2 << 8)], None)):
        p, _, _ = _fixed_anchor_samples(rel, None, [0, 0, 0.5], 50, anchors=anchors, n_obj=3,
                                        anchor_poses=[(0, 0, 0, 0), (0.5, 0, 0, 0)],
                                        poly=((-1, -1), (1, -1), (1, 1), (-1, 1)))
        assert np.array_equal(p, free)


# --------------------------------------------------------------------------- articulated parts

# One prismatic part: axis (0.6, 0, 0.8) (a unit vector with a vertical
# component, so a dropped or swapped axis component shows), q in [0, 1], inside
# support centred at (0.2, -0.1) on z = 0.3, half extents (0.3, 0.15), yaw 0.5.
_PART = [0.6, 0.0, 0.8, 0.0, 1.0, 0.2, -0.1, 0.3, 0.3, 0.15, 0.5, 0.0]


def _inside_batch(n, ratio, q):
    return tiny_batch([[(0.0, 0.0, 0.0, 0.05)], [(0.0, 0.0, 0.0, 0.05)]], n_cand=n,
                      rel=[0, synth.REL_INSIDE | (0 << 8)], relp=[[0.05, 0.2, 0.0, 0.0], [0.0, 0.0, ratio, 0.0]],
                      parts=[_PART], part_q=np.asarray(q, np.float32).reshape(n, 1))


def test_inside_places_on_the_moved_shrunk_support():
    """INSIDE (Sec. IV-F 'inside'): the position is uniform in the part's
    support rectangle moved by q * axis and shrunk by e = ratio * min(Hx, Hy)
    (tiny_batch objects have Hx = Hy = Hz = 0.1, so e = 0.05 at ratio 0.5),
    turned by the part's yaw; z = the moved floor + Hz; accepted at once."""
    n = 4000
    q = np.random.default_rng(0).uniform(0.0, 1.0, n).astype(np.float32)
    b = _inside_batch(n, 0.5, q)
    p, ok, band = oracle.sample_poses(b, seed=11)
    assert ok.all() and not band.any()
    p = p.reshape(n, 2, 4)[:, 1]
    qd = q.astype(np.float64)
    cx, cy, cz = 0.2 + 0.6 * qd, -0.1 + 0.0 * qd, 0.3 + 0.8 * qd
    yaw = np.float32(0.5)
    local = Rotation.from_euler("z", -float(yaw)).apply(np.stack([p[:, 0] - cx, p[:, 1] - cy, 0 * cx], 1))
    assert np.abs(local[:, 0]).max() <= 0.25 + 1e-9 and np.abs(local[:, 1]).max() <= 0.10 + 1e-9
    assert stats.kstest(local[:, 0] / 0.25, stats.uniform(-1, 2).cdf).pvalue > 1e-3
    assert stats.kstest(local[:, 1] / 0.10, stats.uniform(-1, 2).cdf).pvalue > 1e-3
    assert np.allclose(p[:, 2], cz + np.float32(0.1), atol=1e-7)
    # an erosion beyond the half extents leaves the moved centre
    p2, ok2, _ = oracle.sample_poses(_inside_batch(n, 4.0, q), seed=11)
    p2 = p2.reshape(n, 2, 4)[:, 1]
    assert ok2.all() and np.allclose(p2[:, 0], cx, atol=1e-7) and np.allclose(p2[:, 1], cy, atol=1e-7)


def test_inside_naming_a_missing_part_samples_free():
    """An INSIDE object whose part index is not a part of its template is
    sampled with the draws of a free object."""
    n = 64
    q = np.full(n, 0.5, np.float32)
    free = tiny_batch([[(0.0, 0.0, 0.0, 0.05)], [(0.0, 0.0, 0.0, 0.05)]], n_cand=n, parts=[_PART],
                      part_q=q.reshape(n, 1))
    bad = tiny_batch([[(0.0, 0.0, 0.0, 0.05)], [(0.0, 0.0, 0.0, 0.05)]], n_cand=n,
                     rel=[0, synth.REL_INSIDE | (1 << 8)], parts=[_PART], part_q=q.reshape(n, 1))
    pf, _, _ = oracle.sample_poses(free, seed=4)
    pb, _, _ = oracle.sample_poses(bad, seed=4)
    assert np.array_equal(pf, pb)


def test_part_boxes_move_with_their_joint():
    """Translation invariance: a box of part j at joint value q is the static
    box with its centre moved by q * axis_j. Two parts with different axes and
    values (a swapped part index or value shows) and a static box that must
    not move; the static-box distance itself is pinned above."""
    parts = [[0.6, 0.8, 0.0, 0.0, 1.0, 0, 0, 0, 0.1, 0.1, 0, 0], [0.0, 0.0, 1.0, -1.0, 1.0, 0, 0, 0, 0.1, 0.1, 0, 0]]
    boxes = [[0.1, 0.0, 0.2, 0, 0, 0, 0.3826834, 0.9238795, 0.1, 0.2, 0.05, 0],
             [-0.3, 0.2, 0.1, 0, 0.2, 0.1, 0.0, 0.9746794, 0.05, 0.1, 0.1, 0],
             [0.5, -0.5, 0.0, 0, 0, 0, 0, 1, 0.2, 0.2, 0.2, 0]]
    obb_part = [1, 0, -1]
    q = np.array([[0.35, -0.4], [0.9, 0.25], [0.0, 0.0]], np.float32)
    obj = [[(0.0, 0.0, 0.0, 0.05), (0.05, 0.02, 0.0, 0.03)]]
    poses = synth.random_poses(tiny_batch(obj, n_cand=3), seed=3, spread=0.5)
    moving = tiny_batch(obj, obbs=boxes, n_cand=3, parts=parts, obb_part=obb_part, part_q=q)
    _, md, _ = oracle.collide(moving, poses)
    for c in range(3):
        moved = np.array(boxes, np.float64)
        for i, j in enumerate(obb_part):
            if j >= 0:
                moved[i, :3] += np.float64(q[c, j]) * np.array(parts[j][:3], np.float32)
        ref = [oracle.sphere_obb(oracle.sphere_world(s, poses[c]), moved[i].astype(np.float32))
               for s in obj[0] for i in range(3)]
        # the moved centres are rounded to FP32 in the reference: 1e-7 slack
        assert abs(md[c] - min(ref)) <= 1e-6, (c, md[c], min(ref))
    # the joint values matter: candidates 0 and 1 differ from the unmoved boxes
    _, md_static, _ = oracle.collide(tiny_batch(obj, obbs=boxes, n_cand=3), poses)
    assert md[2] == md_static[2] and md[0] != md_static[0] and md[1] != md_static[1]


def test_sample_parts_counter_and_range():
    """Joint values: uniform in [qmin, qmax] from the Philox counter
    (c, 0xFFFF0000 + j, 0, 0) (pinned to numpy's Philox through the shared
    round code above); slots past a template's part count stay 0."""
    b = synth.cabinet(seed=1, n_templates=6, cand_per_template=400)
    q = oracle.sample_parts(b, seed=9)
    nparts = np.diff(b.tmpl_part_off)[b.cand_template()]
    for c in (0, 5, 1234, b.n_cand - 1):
        for j in range(q.shape[1]):
            if j >= nparts[c]:
                assert q[c, j] == 0.0
                continue
            u0 = oracle.uniform4(9, c, 0xFFFF0000 + j, 0, 0)[0]
            assert abs(q[c, j] - np.float64(np.float32(0.35)) * u0) < 1e-15
    live = q[:, :2].ravel()
    assert live.min() >= 0.0 and live.max() < np.float32(0.35)
    assert stats.kstest(live / np.float64(np.float32(0.35)), stats.uniform(0, 1).cdf).pvalue > 1e-3
    act = np.array([3, 7], np.int32)
    qa = oracle.sample_parts(b, seed=9, active=act)
    assert np.array_equal(qa[act], q[act]) and not np.delete(qa, act, axis=0).any()


# --------------------------------------------------------------------------- world meshes


def test_point_triangle_closed_forms():
    """Over the interior: the height above the plane; beyond a vertex: the
    distance to it; beside an edge: the distance to that edge's line; a
    collinear (zero-area) triangle is the segment between its extremes."""
    a, b, c = np.array([0.0, 0, 0]), np.array([2.0, 0, 0]), np.array([0.0, 1.0, 0])
    assert oracle.point_triangle([0.3, 0.2, -0.7], a, b, c) == pytest.approx(0.7, abs=1e-15)
    assert oracle.point_triangle([-1.0, -1.0, 1.0], a, b, c) == pytest.approx(math.sqrt(3), abs=1e-15)
    assert oracle.point_triangle([1.0, -0.5, 0.0], a, b, c) == pytest.approx(0.5, abs=1e-15)
    # beside the hypotenuse b-c (line x + 2y = 2): distance |x + 2y - 2| / sqrt(5)
    p = np.array([1.5, 1.0, 0.25])
    assert oracle.point_triangle(p, a, b, c) == pytest.approx(math.hypot(1.5 / math.sqrt(5), 0.25), abs=1e-14)
    assert oracle.point_triangle([3.0, 1.0, 0.0], a, b, [1.0, 0, 0]) == pytest.approx(math.sqrt(2), abs=1e-15)


def test_point_triangle_brute_force():
    """Against the minimum over a dense barycentric grid of the triangle (a
    brute-force distance: never below the true one, above it by at most the
    grid's spacing), on random triangles and points."""
    rng = np.random.default_rng(3)
    k = 200
    s, t = np.meshgrid(np.arange(k + 1) / k, np.arange(k + 1) / k)
    keep = s + t <= 1
    s, t = s[keep], t[keep]
    for _ in range(40):
        a, b, c = rng.normal(size=(3, 3))
        pts = a + s[:, None] * (b - a) + t[:, None] * (c - a)
        spacing = max(np.linalg.norm(b - a), np.linalg.norm(c - a)) / k
        p = rng.normal(size=3) * 1.5
        d = oracle.point_triangle(p, a, b, c)
        brute = np.min(np.linalg.norm(pts - p, axis=1))
        assert d <= brute + 1e-12 and brute - d <= spacing


def test_box_mesh_distance_is_the_box_sdf():
    """The distance to the 12-triangle surface of a box equals the box's SDF
    (pinned above) outside it and minus the SDF inside it."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        q = Rotation.random(random_state=rng)
        c, h = rng.uniform(-1, 1, 3), rng.uniform(0.05, 0.5, 3)
        box = np.concatenate([c, [0], q.as_quat(), h, [0]]).astype(np.float32)
        # the box from the rounded float32 values both sides see
        cb, qb, hb = box[:3].astype(np.float64), box[4:8].astype(np.float64), box[8:11].astype(np.float64)
        tris = synth.box_mesh(cb, Rotation.from_quat(qb).as_matrix(), hb).astype(np.float32)
        for p in rng.uniform(-1.5, 1.5, (10, 3)):
            sdf = oracle.sphere_obb(np.concatenate([p, [0.0]]), box)
            d = min(oracle.sphere_triangle(np.concatenate([p, [0.0]]), t) for t in tris)
            assert d == pytest.approx(abs(sdf), abs=2e-6)


def test_collide_counts_the_nearest_triangle():
    """A one-sphere object over a triangle: min_dist is the plane height minus
    r (closed form), a collision once the sphere dips through the surface, and
    triangles only count for objects >= first_new."""
    tri = [[0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0]]
    b = tiny_batch([[(0.0, 0.0, 0.0, 0.05)], [(0.0, 0.0, 0.0, 0.05)]], n_cand=3)
    b.tmpl_tri_off, b.tri = np.array([0, 1], np.int32), np.array(tri, np.float32)
    poses = np.array([[5, 5, 5, 0], [0.2, 0.2, 0.30, 1.0],
                      [5, 5, 5, 0], [0.2, 0.2, 0.03, 0.0],
                      [0.2, 0.2, 0.03, 0.0], [-5, -5, 5, 0]], np.float32)
    col, md, _ = oracle.collide(b, poses)
    assert md[0] == pytest.approx(np.float64(np.float32(0.30)) - np.float64(np.float32(0.05)), abs=1e-12)
    assert col[1] == 1 and md[1] == pytest.approx(np.float64(np.float32(0.03)) - np.float64(np.float32(0.05)))
    col2, md2, _ = oracle.collide(b, poses, first_new=1)
    assert col2[2] == 0 and md2[2] > 1.0  # object 0 dips through the triangle but is not new
