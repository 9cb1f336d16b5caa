"""Articulated parts (prismatic joints such as drawers, and the INSIDE
relation of Sec. IV-F) on the GPU against the FP64 oracle, through the C ABI.

Joint values are inputs drawn by the seeded generator (the same numbers for
both sides); sc_sample_parts is compared with the oracle's own draw. The
contract is the one of the other parity tests: decisions agree outside the
1e-5 m band, distances and poses within 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from scenes import tiny_batch
from test_gpu_parity import check_collide, check_samples, pose_rows

pytestmark = pytest.mark.gpu

TOL_POSE = 1e-5


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


def cabinet_poses(b, seed):
    """Object poses spread over the cabinet and its open drawers (float32):
    x in [-0.7, 0.35], y in [-0.4, 0.4], z in [0, 1.0], yaw uniform."""
    rng = np.random.default_rng(seed)
    n = b.n_poses()
    p = np.stack([rng.uniform(-0.7, 0.35, n), rng.uniform(-0.4, 0.4, n), rng.uniform(0.0, 1.0, n),
                  rng.uniform(0, 2 * np.pi, n)], 1)
    return p.astype(np.float32)


def test_sample_parts_matches_oracle(sc, ctx):
    """Joint values: the same Philox draw on both sides; FP32 against FP64
    within a few ulps of the range; untouched slots and unlisted candidates
    keep what the buffer held."""
    b = synth.cabinet(seed=2, n_templates=20, cand_per_template=33)
    db = sc.DeviceBatch(b)
    db.t["part_q"].fill_(-7.0)
    act = np.arange(0, b.n_cand, 3, dtype=np.int32)
    q = sc.sample_parts(ctx, db, seed=17, active=torch.from_numpy(act).cuda()).cpu().numpy()
    ctx.synchronize()
    oq = oracle.sample_parts(b, seed=17, active=act)
    nparts = np.diff(b.tmpl_part_off)[b.cand_template()]
    slot = np.arange(q.shape[1])[None, :] < nparts[:, None]
    listed = np.zeros(b.n_cand, bool)
    listed[act] = True
    live = slot & listed[:, None]
    assert np.max(np.abs(q[live] - oq[live])) <= 1e-7
    assert np.all(q[~live] == -7.0)


@pytest.mark.parametrize("seed", [0, 1])
def test_sample_inside_matches_oracle(sc, ctx, seed):
    """Every object of the cabinet workload, INSIDE objects included, from the
    same joint values."""
    b = synth.cabinet(seed=seed, n_templates=24, cand_per_template=16)
    db = sc.DeviceBatch(b)
    gp, gok, gband = sc.sample_poses(ctx, db, seed=seed + 3)
    ctx.synchronize()
    op, ook, oband = oracle.sample_poses(b, seed=seed + 3)
    band, d = check_samples(gp, gok, gband, op, ook, oband)
    rows = pose_rows(b, np.nonzero(~band)[0])
    assert d[rows].max() <= TOL_POSE


@pytest.mark.parametrize("decide", [0, 1])
def test_collide_moving_boxes_matches_oracle(sc, ctx, decide):
    """Spheres against boxes that move with their drawer, both collision
    modes: (a) few objects at poses spread over the open drawers; (b) the
    oracle's collision-free scenes with the drawers moved to new joint
    values, so resting objects now meet walls and floors."""
    cfg = (0, 0, 0, 0, 1) if decide else None
    few = synth.cabinet(seed=4, n_templates=16, cand_per_template=24, counter_range=(1, 1), inside_per_drawer=1)
    full = synth.cabinet(seed=4, n_templates=16, cand_per_template=24)
    p, v, _, _ = oracle.generate(full, seed=8, max_retries=10)
    act = np.nonzero(v)[0].astype(np.int32)
    moved = synth.cabinet(seed=4, n_templates=16, cand_per_template=24)
    moved.part_q[:] = np.random.default_rng(1).uniform(0, 0.35, moved.part_q.shape).astype(np.float32)
    cases = [(few, cabinet_poses(few, 5), None), (full, np.nan_to_num(p).astype(np.float32), act),
             (moved, np.nan_to_num(p).astype(np.float32), act)]
    rates = []
    for b, poses, active in cases:
        db = sc.DeviceBatch(b)
        at = None if active is None else torch.from_numpy(active).cuda()
        gcol, gmd, gband = sc.collide(ctx, db, torch.from_numpy(poses).cuda(), active=at, config=cfg)
        ctx.synchronize()
        ocol, omd, oband = oracle.collide(b, poses, active=active)
        if decide:
            band = gband.cpu().numpy().astype(bool) | oband.astype(bool)
            assert band.mean() <= 0.01
            assert np.array_equal(gcol.cpu().numpy()[~band], ocol[~band])
        else:
            check_collide(gcol, gmd, gband, ocol, omd, oband)
        rates.append(ocol.mean())
    assert rates[1] == 0.0 and 0.2 < rates[2] < 0.95, rates


def test_part_arrays_validated(sc, ctx):
    """A batch with parts but no joint values is refused on the host; a box
    or an INSIDE object naming a part its template lacks latches device
    code 8 (the box stays put, the object is sampled free)."""
    b = synth.cabinet(seed=1, n_templates=2, cand_per_template=4)
    db = sc.DeviceBatch(b)
    db.c.part_q = None
    with pytest.raises(sc.SceniError):
        sc.sample_poses(ctx, db, seed=1)
    part = [[1.0, 0.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.2, 0.2, 0.0, 0.0]]
    bad_box = tiny_batch([[(0, 0, 0, 0.01)]], obbs=[[0.5, 0, 0, 0, 0, 0, 0, 1, 0.1, 0.1, 0.1, 0]], n_cand=2,
                         parts=part, obb_part=[3])
    dbb = sc.DeviceBatch(bad_box)
    col, md, band = sc.collide(ctx, dbb, dbb.new_poses())
    with pytest.raises(sc.SceniError) as ei:
        ctx.synchronize()
    assert "device error code 8" in str(ei.value)
    # and the candidates carry no verdict: NaN, banded, not colliding
    assert torch.isnan(md).all() and (band == 1).all() and (col == 0).all()
    bad_rel = tiny_batch([[(0, 0, 0, 0.01)]] * 2, n_cand=2, rel=[0, synth.REL_INSIDE | (2 << 8)], parts=part)
    sc.sample_poses(ctx, sc.DeviceBatch(bad_rel), seed=1)
    with pytest.raises(sc.SceniError) as ei:
        ctx.synchronize()
    assert "device error code 8" in str(ei.value)
    ctx.synchronize()


def test_part_count_limit_refused(sc, ctx):
    """More than 16 parts in a template (max_parts > 16) is refused on the host."""
    part = [[1.0, 0.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.2, 0.2, 0.0, 0.0]] * 17
    b = tiny_batch([[(0, 0, 0, 0.01)]], n_cand=2, parts=part)
    with pytest.raises(sc.SceniError):
        sc.sample_poses(ctx, sc.DeviceBatch(b), seed=1)
    ctx.synchronize()


def test_random_parts_rotated_boxes_match_oracle(sc, ctx):
    """Parts with random unit axes (vertical components included), yawed
    inside supports and rotated boxes owned by them, random joint values per
    candidate: INSIDE sampling and whole-scene collision against the oracle."""
    rng = np.random.default_rng(12)
    n_cand, n_parts = 400, 3
    parts = []
    for j in range(n_parts):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        parts.append([*ax, -0.2, 0.3, rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.0, 0.4),
                      rng.uniform(0.1, 0.3), rng.uniform(0.1, 0.3), rng.uniform(-np.pi, np.pi), 0.0])
    boxes = synth.random_obbs(rng, 6)
    obb_part = [0, 1, 2, 0, -1, 2]
    objects = [[(0.0, 0.0, 0.0, 0.05), (0.04, 0.0, 0.02, 0.03)] for _ in range(5)]
    rel = [0, synth.REL_INSIDE | (0 << 8), synth.REL_INSIDE | (1 << 8), synth.REL_INSIDE | (2 << 8),
           synth.REL_ON_TOP | (1 << 8)]
    relp = [[0.05, 0.2, 0.0, 0.0], [0, 0, 0.5, 0], [0, 0, 1.0, 0], [0, 0, 0.0, 0], [0.05, 0.2, 0.0, 0.0]]
    q = rng.uniform(-0.2, 0.3, (n_cand, n_parts)).astype(np.float32)
    b = tiny_batch(objects, obbs=boxes, n_cand=n_cand, rel=rel, relp=relp, parts=parts, obb_part=obb_part, part_q=q)
    db = sc.DeviceBatch(b)
    gp, gok, gband = sc.sample_poses(ctx, db, seed=21)
    ctx.synchronize()
    op, ook, oband = oracle.sample_poses(b, seed=21)
    band, d = check_samples(gp, gok, gband, op, ook, oband)
    assert d[pose_rows(b, np.nonzero(~band)[0])].max() <= TOL_POSE
    poses = op.astype(np.float32)
    gcol, gmd, gcb = sc.collide(ctx, db, torch.from_numpy(poses).cuda())
    ctx.synchronize()
    ocol, omd, ocb = oracle.collide(b, poses)
    check_collide(gcol, gmd, gcb, ocol, omd, ocb)
    assert 0.05 < ocol.mean() < 1.0
