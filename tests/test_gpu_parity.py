"""GPU (FP32, CUDA) against the FP64 oracle, through the C ABI.

Contract: collision / acceptance decisions agree bit-exactly outside the
1e-5 m decision band (a candidate either side flags as band is excluded and
counted); distances agree within 1e-5 m; poses agree within 1e-5 m / 1e-5 rad.
Inputs are seeded synthetic batches; no expected value comes from the GPU.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from scenes import tiny_batch

pytestmark = pytest.mark.gpu

TOL_DIST = 1e-5   # metres: distance agreement (the decision band width)
TOL_POSE = 1e-5   # metres / radians: sampled pose agreement
FLT_MAX = np.finfo(np.float32).max


@pytest.fixture(scope="module")
def sc():
    import paper_2512_16896_b300 as sc
    from paper_2512_16896_b300 import build
    build.build()
    return sc


@pytest.fixture(scope="module")
def ctx(sc):
    c = sc.Context()
    yield c
    c.close()


def check_samples(gp, gok, gband, op, ook, oband, active_pose_rows=None, max_band_frac=0.01):
    gp = gp.cpu().numpy().astype(np.float64)
    gok, gband = gok.cpu().numpy(), gband.cpu().numpy()
    band = gband.astype(bool) | oband.astype(bool)
    assert band.mean() <= max_band_frac, band.mean()
    assert np.array_equal(gok[~band], ook[~band])
    rows = slice(None) if active_pose_rows is None else active_pose_rows
    d = np.abs(gp[rows] - op[rows])
    d[:, 3] = np.minimum(d[:, 3], 2 * np.pi - d[:, 3])
    return band, d


def check_collide(gcol, gmd, gband, ocol, omd, oband, max_band_frac=0.01):
    gcol, gmd, gband = gcol.cpu().numpy(), gmd.cpu().numpy().astype(np.float64), gband.cpu().numpy()
    band = gband.astype(bool) | oband.astype(bool)
    assert band.mean() <= max_band_frac, band.mean()
    assert np.array_equal(gcol[~band], ocol[~band]), np.nonzero(gcol[~band] != ocol[~band])
    fmax_g, fmax_o = gmd == FLT_MAX, omd >= FLT_MAX * 0.999
    assert np.array_equal(fmax_g, fmax_o)
    assert np.max(np.abs(gmd[~fmax_g] - omd[~fmax_g]), initial=0.0) <= TOL_DIST
    return band


def pose_rows(batch, cands):
    """CSR pose rows of the listed candidates (oracle's own layout walk)."""
    offs = oracle.pose_offsets(batch)
    nobj = np.diff(batch.tmpl_obj_off)[batch.cand_template()]
    return np.concatenate([np.arange(offs[c], offs[c] + nobj[c]) for c in cands])


# --------------------------------------------------------------------------- sampling


@pytest.mark.parametrize("make,seed", [
    (lambda: synth.tabletop(seed=0, n_cand=1024), 0),
    (lambda: synth.shelf(seed=1, n_cand=300, n_obj=32, n_sph=8, n_obb=0), 1),
    (lambda: synth.ragged(seed=2, n_templates=48, cand_per_template=7), 2),
])
def test_sample_all_objects(sc, ctx, make, seed):
    b = make()
    db = sc.DeviceBatch(b)
    gp, gok, gband = sc.sample_poses(ctx, db, seed=seed)
    ctx.synchronize()
    op, ook, oband = oracle.sample_poses(b, seed=seed)
    band, d = check_samples(gp, gok, gband, op, ook, oband)
    rows = pose_rows(b, np.nonzero(~band)[0])
    assert d[rows].max() <= TOL_POSE, d[rows].max(axis=0)


@pytest.mark.parametrize("seed", [3, 4])
def test_sample_relation_set(sc, ctx, seed):
    """The full relation set of Sec. IV-F (on-top, next-to, directional in the
    world and the anchor's frame with finite and open radii, middle of 2..4
    anchors, face-to), chained through earlier objects' poses."""
    b = synth.hard(seed=seed, n_templates=48, cand_per_template=16)
    kinds = b.obj_rel & 0xF
    assert (kinds == synth.REL_DIRECTIONAL).any() and (kinds == synth.REL_MIDDLE).any()
    assert (b.obj_rel & synth.REL_FACE_TO).any() and (b.obj_rel & synth.REL_LOCAL).any()
    db = sc.DeviceBatch(b)
    gp, gok, gband = sc.sample_poses(ctx, db, seed=seed)
    ctx.synchronize()
    op, ook, oband = oracle.sample_poses(b, seed=seed)
    band, d = check_samples(gp, gok, gband, op, ook, oband, max_band_frac=0.02)
    # a face-to yaw is the direction to the reference: compare the aimed point,
    # i.e. the yaw difference times the distance to the reference (metres)
    offs, t_of = oracle.pose_offsets(b), b.cand_template()
    for c in range(b.n_cand):
        o0 = b.tmpl_obj_off[t_of[c]]
        for k in range(b.n_obj_of(t_of[c])):
            rel = int(b.obj_rel[o0 + k])
            if rel & synth.REL_FACE_TO and (rel & 0xF) != synth.REL_ON_TOP:
                row, ref = offs[c] + k, offs[c] + ((rel >> 8) & 0xFF)
                d[row, 3] *= np.hypot(*(op[ref, :2] - op[row, :2]))
    rows = pose_rows(b, np.nonzero(~band)[0])
    assert d[rows].max() <= TOL_POSE, d[rows].max(axis=0)
    assert 0.05 < ook.mean() < 0.95


def test_relation_arrays_validated(sc, ctx):
    """A batch with anchors but no anchor offsets is refused on the host; a
    MIDDLE object whose anchors name itself latches a device error."""
    b = synth.hard(seed=3, n_templates=4, cand_per_template=4)
    db = sc.DeviceBatch(b)
    db.c.obj_anchor_off = None
    with pytest.raises(sc.SceniError):
        sc.sample_poses(ctx, db, seed=1)
    rel = [0, 0, synth.REL_MIDDLE]
    bad = tiny_batch([[(0, 0, 0, 0.01)]] * 3, n_cand=4, rel=rel, anchors=[[], [], [0, 2]])
    sc.sample_poses(ctx, sc.DeviceBatch(bad), seed=1)
    with pytest.raises(sc.SceniError) as ei:
        ctx.synchronize()
    assert ei.value.status == 6
    ctx.synchronize()


def test_sample_active_list_retry_and_object_range(sc, ctx):
    """A subset of candidates, retry index 3, objects 2..5 only, with objects
    0..1 sampled by an earlier call on each side."""
    b = synth.shelf(seed=3, n_cand=200, n_obj=12, n_sph=4, n_obb=0)
    db = sc.DeviceBatch(b)
    act = np.sort(np.random.default_rng(0).choice(b.n_cand, 77, replace=False)).astype(np.int32)
    gp, _, _ = sc.sample_poses(ctx, db, seed=9, retry=1, first_obj=0, n_obj=2)
    gp, gok, gband = sc.sample_poses(ctx, db, seed=9, retry=3, first_obj=2, n_obj=4,
                                     active=torch.from_numpy(act).cuda(), poses=gp)
    ctx.synchronize()
    op, _, _ = oracle.sample_poses(b, seed=9, retry=1, first_obj=0, n_obj=2)
    op, ook, oband = oracle.sample_poses(b, seed=9, retry=3, first_obj=2, n_obj=4, active=act, poses=op)
    band, d = check_samples(gp, gok, gband, op, ook, oband)
    rows = pose_rows(b, act[~band])
    assert d[rows].max() <= TOL_POSE


def test_sample_erosion_and_many_attempts(sc, ctx):
    b = synth.ragged(seed=4, n_templates=16, cand_per_template=16)
    b.obj_rel_param[:, 2] = 0.8  # ratio_on_support
    db = sc.DeviceBatch(b)
    for K in (1, 40):  # single attempt; attempts spanning two warp chunks
        gp, gok, gband = sc.sample_poses(ctx, db, seed=11, max_attempts=K)
        op, ook, oband = oracle.sample_poses(b, seed=11, max_attempts=K)
        band, d = check_samples(gp, gok, gband, op, ook, oband, max_band_frac=0.05)
        rows = pose_rows(b, np.nonzero(~band)[0])
        assert d[rows].max() <= TOL_POSE
        if K == 1:
            assert ook.mean() < 1.0  # rejections happen


# --------------------------------------------------------------------------- collision


@pytest.mark.parametrize("make", [
    lambda: synth.tabletop(seed=0, n_cand=1024),
    lambda: synth.shelf(seed=1, n_cand=97, n_obj=32, n_sph=64, n_obb=20),
    lambda: synth.ragged(seed=2, n_templates=24, cand_per_template=3, obj_range=(2, 40), sph_range=(1, 130)),
])
def test_collide_random_poses(sc, ctx, make):
    """Same float32 poses into both sides (no sampling involved)."""
    b = make()
    db = sc.DeviceBatch(b)
    poses = synth.random_poses(b, seed=5, spread=0.5)
    gcol, gmd, gband = sc.collide(ctx, db, torch.from_numpy(poses).cuda())
    ctx.synchronize()
    ocol, omd, oband = oracle.collide(b, poses)
    check_collide(gcol, gmd, gband, ocol, omd, oband)


@pytest.mark.parametrize("make", [
    lambda: synth.tabletop(seed=0, n_cand=1024),
    lambda: synth.shelf(seed=1, n_cand=97, n_obj=32, n_sph=64, n_obb=20),
    lambda: synth.shelf(seed=3, n_cand=64, n_obj=12, n_sph=100, n_obb=6),
    lambda: synth.ragged(seed=2, n_templates=24, cand_per_template=3, obj_range=(2, 40), sph_range=(1, 130)),
])
def test_collide_decide_only(sc, ctx, make):
    """Decide-only mode (Sec. IV-D, a yes/no per candidate): the decision and
    band agree with the oracle; min_dist is above the band (FLT_MAX when no
    pair was close enough to evaluate) for a clear candidate, below -band for
    a certain collision, and the exact minimum (bit-identical to the
    exact-minimum mode) inside the band."""
    b = make()
    db = sc.DeviceBatch(b)
    poses = synth.random_poses(b, seed=5, spread=0.5)
    pt = torch.from_numpy(poses).cuda()
    ecol, emd, eband = (x.cpu().numpy() for x in sc.collide(ctx, db, pt))
    dcol, dmd, dband = (x.cpu().numpy() for x in sc.collide(ctx, db, pt, config=(0, 0, 0, 0, 1)))
    ctx.synchronize()
    ocol, omd, oband = oracle.collide(b, poses)
    band = dband.astype(bool) | oband.astype(bool)
    assert band.mean() <= 0.01
    assert np.array_equal(dcol[~band], ocol[~band])
    clear = ~band & (ocol == 0)
    assert np.all(dmd[clear] > 1e-5)
    hit = ~band & (ocol == 1)
    assert np.all(dmd[hit] < -1e-5)
    inside = eband.astype(bool) & (np.abs(emd) < 0.999e-5)
    assert np.array_equal(dband[inside], eband[inside]) and np.array_equal(dmd[inside], emd[inside])


@pytest.mark.parametrize("mode", [0, 1])
def test_collide_boxes_near_and_far(sc, ctx, mode):
    """World boxes at every range from the objects: most candidates clear
    (the minimum is the distance to the nearest box or pair, including boxes
    whose distance only a later pass of the per-(object, box) ball cull
    reaches), some grazing, some inside a box."""
    rng = np.random.default_rng(31)
    objs = [[(float(x), float(y), float(z), float(r)) for x, y, z, r in
             np.c_[rng.uniform(-0.08, 0.08, (n, 3)), rng.uniform(0.01, 0.04, n)]] for n in (40, 7, 70, 1, 33)]
    obbs = []
    for i in range(9):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        c = rng.uniform([-1.5, -1.5, 0.0], [1.5, 1.5, 1.0])
        obbs.append([*c, 0, *q, *rng.uniform(0.02, 0.4, 3), 0])
    b = tiny_batch(objs, obbs=obbs, n_cand=600)
    poses = synth.random_poses(b, seed=32, spread=1.6)
    g = sc.collide(ctx, sc.DeviceBatch(b), torch.from_numpy(poses).cuda(), config=(0, 0, 0, 0, mode))
    ctx.synchronize()
    ocol, omd, oband = oracle.collide(b, poses)
    gcol, gmd, gband = (x.cpu().numpy() for x in g)
    band = gband.astype(bool) | oband.astype(bool)
    assert np.array_equal(gcol[~band], ocol[~band])
    assert 0.2 < ocol.mean() < 0.8, ocol.mean()
    if mode == 0:
        check_collide(*g, ocol, omd, oband)
    else:
        assert np.all(gmd[~band & (ocol == 0)] > 1e-5) and np.all(gmd[~band & (ocol == 1)] < -1e-5)


@pytest.mark.parametrize("first_new", [0, 1, 5, 7, 8, 100])
def test_collide_first_new(sc, ctx, first_new):
    b = synth.tabletop(seed=6, n_cand=333)
    db = sc.DeviceBatch(b)
    poses = synth.random_poses(b, seed=7, spread=0.4)
    g = sc.collide(ctx, db, torch.from_numpy(poses).cuda(), first_new=first_new)
    ctx.synchronize()
    o = oracle.collide(b, poses, first_new=first_new)
    check_collide(*g, *o)
    if first_new >= 8:
        assert np.all(g[1].cpu().numpy() == FLT_MAX) and not g[0].any()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("first_new", [0, 3, 9])
def test_collide_offset_spheres_culls(sc, ctx, mode, first_new):
    """Objects whose spheres sit far from the object origin (the bounding
    balls are centred on the origin, so their radii are large and lopsided),
    objects of one sphere, of many spheres and world boxes, in both modes and
    with earlier objects already placed: the per-(object, box) and
    per-object-pair ball culls must not drop a pair that decides."""
    rng = np.random.default_rng(41)
    objs = []
    for n in (1, 90, 5, 33, 1, 140, 12, 64, 2, 40, 7, 20):
        off = rng.uniform(-0.25, 0.25, 3)
        c = off + rng.uniform(-0.05, 0.05, (n, 3))
        objs.append([(float(x), float(y), float(z), float(r)) for (x, y, z), r in zip(c, rng.uniform(0.005, 0.05, n))])
    obbs = []
    for i in range(5):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        obbs.append([*rng.uniform([-0.8, -0.8, 0.0], [0.8, 0.8, 0.5]), 0, *q, *rng.uniform(0.02, 0.3, 3), 0])
    b = tiny_batch(objs, obbs=obbs, n_cand=500)
    poses = synth.random_poses(b, seed=42, spread=0.9)
    g = sc.collide(ctx, sc.DeviceBatch(b), torch.from_numpy(poses).cuda(), first_new=first_new,
                   config=(0, 0, 0, 0, mode))
    ctx.synchronize()
    ocol, omd, oband = oracle.collide(b, poses, first_new=first_new)
    gcol, gmd, gband = (x.cpu().numpy() for x in g)
    band = gband.astype(bool) | oband.astype(bool)
    assert np.array_equal(gcol[~band], ocol[~band])
    assert 0.05 < ocol.mean() < 0.95, ocol.mean()
    if mode == 0:
        check_collide(*g, ocol, omd, oband)
    else:
        assert np.all(gmd[~band & (ocol == 0)] > 1e-5) and np.all(gmd[~band & (ocol == 1)] < -1e-5)


@pytest.mark.parametrize("cfg", [(128, 1, 8, 1), (1024, 2, 64, 1), (512, 4, 4096, 2), (256, 4, 256, 4), (96 * 4, 2, 24, 3)])
def test_collide_configs_bit_identical(sc, ctx, cfg):
    """Every launch shape reduces the same per-pair values: min_dist bit-identical."""
    b = synth.ragged(seed=8, n_templates=20, cand_per_template=4)
    db = sc.DeviceBatch(b)
    poses = torch.from_numpy(synth.random_poses(b, seed=9)).cuda()
    ref = sc.collide(ctx, db, poses)
    got = sc.collide(ctx, db, poses, config=cfg)
    ctx.synchronize()
    assert torch.equal(ref[1], got[1]) and torch.equal(ref[0], got[0]) and torch.equal(ref[2], got[2])


@pytest.mark.parametrize("make,first_new", [
    (lambda: synth.shelf(seed=12, n_cand=300, n_obj=12, n_sph=40, n_obb=6), 0),
    (lambda: synth.ragged(seed=13, n_templates=24, cand_per_template=5), 2),
    (lambda: synth.tabletop(seed=14, n_cand=200), 0),
])
@pytest.mark.parametrize("mode", [0, 1])
def test_collide_bulk_staging_bit_identical(sc, ctx, make, first_new, mode):
    """The local spheres copied in one bulk asynchronous copy per candidate
    (stage_bulk = 1) give exactly what per-lane loads give, over consecutive
    candidates of one template and of different ones: every output in
    exact-minimum mode; in decide-only mode, where a candidate stops at
    whichever certain collision its warps meet first, the decision, the band
    and the distance inside the band, and a distance on the right side of
    the band elsewhere."""
    b = make()
    db = sc.DeviceBatch(b)
    poses = torch.from_numpy(synth.random_poses(b, seed=15, spread=0.5)).cuda()
    order = torch.from_numpy(sc.order_by_work(b)).cuda()
    for shape in ((0, 0, 0, 0), (128, 2, 64, 2)):
        ref = sc.collide(ctx, db, poses, active=order, first_new=first_new, config=shape + (mode, 0))
        got = sc.collide(ctx, db, poses, active=order, first_new=first_new, config=shape + (mode, 1))
        ctx.synchronize()
        if mode == 0:
            for x, y in zip(ref, got):
                assert torch.equal(x, y)
            continue
        (rc, rd, rb), (gc, gd, gb) = ref, got
        assert torch.equal(rc, gc) and torch.equal(rb, gb)
        inside = rd.abs() <= 1e-5
        assert torch.equal(rd[inside], gd[inside]) and torch.equal(gd.abs() <= 1e-5, inside)
        assert bool(((gd < -1e-5) == (rd < -1e-5)).all()) and bool(((gd > 1e-5) == (rd > 1e-5)).all())


def test_collide_lpt_active_list_and_empty(sc, ctx):
    b = synth.ragged(seed=10, n_templates=30, cand_per_template=5)
    db = sc.DeviceBatch(b)
    poses = synth.random_poses(b, seed=11)
    order = sc.order_by_work(b)
    g = sc.collide(ctx, db, torch.from_numpy(poses).cuda(), active=torch.from_numpy(order).cuda())
    ctx.synchronize()
    o = oracle.collide(b, poses, active=order)
    check_collide(*g, *o)
    e = sc.collide(ctx, db, torch.from_numpy(poses).cuda(), active=torch.zeros(0, dtype=torch.int32, device="cuda"))
    ctx.synchronize()
    assert e[0].numel() == 0


def test_collide_degenerate_scenes(sc, ctx):
    """One object (no pairs, no world) -> FLT_MAX; exact touching -> band; a
    sphere swallowed by a world box -> collision."""
    one = tiny_batch([[(0, 0, 0, 0.1), (0.05, 0, 0, 0.1)]], n_cand=3)
    g = sc.collide(ctx, sc.DeviceBatch(one), torch.zeros((3, 4), device="cuda"))
    ctx.synchronize()
    assert np.all(g[1].cpu().numpy() == FLT_MAX) and not g[0].any()
    touch = tiny_batch([[(0, 0, 0, 0.125)], [(0, 0, 0, 0.125)]], n_cand=2)
    p = torch.tensor([[0, 0, 0, 0], [0.25, 0, 0, 0], [0, 0, 0, 0], [0.2, 0, 0, 0]], dtype=torch.float32, device="cuda")
    col, md, band = sc.collide(ctx, sc.DeviceBatch(touch), p)
    ctx.synchronize()
    assert band[0].item() == 1 and abs(md[0].item()) <= TOL_DIST
    assert col[1].item() == 1 and md[1].item() == pytest.approx(-0.05, abs=1e-6)
    world = tiny_batch([[(0, 0, 0, 0.1)]], obbs=[[3, 0, 0, 0, 0, 0, 0, 1, 0.5, 0.5, 0.5, 0]], n_cand=2)
    p = torch.tensor([[0, 0, 0, 0], [2.9, 0, 0, 0]], dtype=torch.float32, device="cuda")
    g = sc.collide(ctx, sc.DeviceBatch(world), p)
    o = oracle.collide(world, p.cpu().numpy())
    ctx.synchronize()
    check_collide(*g, *o)


def test_device_error_is_latched_not_faulted(sc, ctx):
    """A batch that under-states max_sph is caught by the kernel's own check:
    the candidate is skipped and sc_ctx_synchronize reports SC_ERR_DEVICE."""
    b = synth.tabletop(seed=0, n_cand=8)
    db = sc.DeviceBatch(b)
    db.c.max_sph = 16
    sc.collide(ctx, db, torch.from_numpy(synth.random_poses(b, seed=1)).cuda())
    with pytest.raises(sc.SceniError) as ei:
        ctx.synchronize()
    assert ei.value.status == 6
    ctx.synchronize()  # cleared


# --------------------------------------------------------------------------- full sizes, sampled


def _sampled_full(sc, ctx, b, seed, n_check, rng_seed, extra=()):
    db = sc.DeviceBatch(b)
    order = torch.from_numpy(sc.order_by_work(b)).cuda()
    gp, gok, gband = sc.sample_poses(ctx, db, seed=seed)
    gcol, gmd, gcb = sc.collide(ctx, db, gp, active=order)
    ctx.synchronize()
    # outputs are in list order; map back to candidate index
    inv = torch.empty_like(order)
    inv[order] = torch.arange(order.numel(), device="cuda", dtype=order.dtype)
    gcol, gmd, gcb = gcol[inv.long()], gmd[inv.long()], gcb[inv.long()]
    pick = np.random.default_rng(rng_seed).choice(b.n_cand, n_check, replace=False)
    pick = np.unique(np.concatenate([pick, list(extra)])).astype(np.int32)
    op, ook, oband = oracle.sample_poses(b, seed=seed, active=pick)
    sel = torch.from_numpy(pick).long().cuda()
    sband, d = check_samples(gp, gok[sel], gband[sel], op, ook, oband, active_pose_rows=pose_rows(b, pick),
                             max_band_frac=0.05)
    nobj = np.diff(b.tmpl_obj_off)[b.cand_template()[pick]]
    keep_rows = np.repeat(~sband, nobj)
    assert d[keep_rows].max(initial=0.0) <= TOL_POSE
    ocol, omd, ocb = oracle.collide(b, op, active=pick)
    band = check_collide(gcol[sel], gmd[sel], gcb[sel], ocol, omd, ocb | sband, max_band_frac=0.05)
    return gcol, gmd


def test_full_shelf_sampled(sc, ctx):
    """65,536 candidates x 32 objects x 64 spheres + 20 boxes, in the launch
    configuration the benchmark uses; 48 random candidates against the oracle."""
    b = synth.shelf(seed=1)
    gcol, gmd = _sampled_full(sc, ctx, b, seed=1, n_check=48, rng_seed=0, extra=(0, b.n_cand - 1))
    assert torch.isfinite(gmd).all()


@pytest.mark.slow
def test_full_ragged_sampled(sc, ctx):
    """4096 templates x 64 candidates (ragged); 64 random candidates plus the
    heaviest template's first candidate against the oracle."""
    b = synth.ragged(seed=2)
    heavy = int(sc.order_by_work(b)[0])
    _sampled_full(sc, ctx, b, seed=2, n_check=64, rng_seed=1, extra=(heavy, 0, b.n_cand - 1))
