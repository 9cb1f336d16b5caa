"""World triangle meshes on the GPU against the FP64 oracle, through the C ABI.

A sphere's distance to a mesh is the unsigned distance from its centre to the
nearest triangle point minus its radius. Contract as in the other parity
tests: decisions agree outside the 1e-5 m band, distances within 1e-5 m.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from scenes import tiny_batch
from test_gpu_parity import check_collide

pytestmark = pytest.mark.gpu


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


def mesh_poses(b, seed):
    """Object poses over the supports and through the clutter (float32):
    x, y in [-1, 1], z in [0.7, 1.15], yaw uniform."""
    rng = np.random.default_rng(seed)
    n = b.n_poses()
    p = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0.7, 1.15, n),
                  rng.uniform(0, 2 * np.pi, n)], 1)
    return p.astype(np.float32)


@pytest.mark.parametrize("decide", [0, 1])
@pytest.mark.parametrize("first_new", [0, 2])
def test_collide_meshes_matches_oracle(sc, ctx, decide, first_new):
    """Few objects through the clutter (triangles decide most outcomes), then
    the oracle's collision-free scenes (none collide)."""
    cfg = (0, 0, 0, 0, 1) if decide else None
    few = synth.meshes(seed=3, n_templates=24, cand_per_template=12, obj_range=(2, 4), sph_range=(4, 24))
    full = synth.meshes(seed=4, n_templates=16, cand_per_template=12)
    p, v, _, _ = oracle.generate(full, seed=5, max_retries=10)
    act = np.nonzero(v)[0].astype(np.int32)
    rates = []
    for b, poses, active in ((few, mesh_poses(few, 1), None), (full, np.nan_to_num(p).astype(np.float32), act)):
        db = sc.DeviceBatch(b)
        at = None if active is None else torch.from_numpy(active).cuda()
        gcol, gmd, gband = sc.collide(ctx, db, torch.from_numpy(poses).cuda(), active=at, first_new=first_new,
                                      config=cfg)
        ctx.synchronize()
        ocol, omd, oband = oracle.collide(b, poses, active=active, first_new=first_new)
        if decide:
            band = gband.cpu().numpy().astype(bool) | oband.astype(bool)
            assert band.mean() <= 0.05  # resting contacts (on-top children) sit at distance ~0
            assert np.array_equal(gcol.cpu().numpy()[~band], ocol[~band])
        else:
            check_collide(gcol, gmd, gband, ocol, omd, oband, max_band_frac=0.05)
        rates.append(ocol.mean())
    assert 0.1 < rates[0] < 0.95 and rates[1] == 0.0, rates


def test_triangle_cases_and_work(sc, ctx):
    """One sphere against single triangles in every Voronoi region (above the
    face, beside each edge, beyond each vertex) and against zero-area
    triangles (collinear, a point): distances within 1e-6 of the oracle; the
    point-triangle distances the kernel reports are at most a ball cull per
    pass (two in exact-minimum mode) and an exact distance per candidate."""
    tris = [[0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0],       # right triangle in z = 0
            [0, 0, 0, 0, 1, 1, 0, 0, 2, 2, 0, 0],       # collinear
            [0.3, 0.3, 0.3, 0, 0.3, 0.3, 0.3, 0, 0.3, 0.3, 0.3, 0]]  # a point
    pts = np.array([[0.2, 0.2, 0.4], [0.5, -0.3, 0.1], [-0.3, 0.4, -0.2], [0.8, 0.8, 0.05], [-0.2, -0.2, 0.3],
                    [1.4, -0.1, 0.2], [-0.1, 1.3, -0.1], [0.6, 0.6, 0.0], [0.35, 0.3, 0.25], [1.5, 1.5, 0.4]])
    for t in tris:
        b = tiny_batch([[(0.0, 0.0, 0.0, 0.01)]], n_cand=len(pts))
        b.tmpl_tri_off, b.tri = np.array([0, 1], np.int32), np.array([t], np.float32)
        poses = np.concatenate([pts, np.zeros((len(pts), 1))], 1).astype(np.float32)
        db = sc.DeviceBatch(b)
        _, gmd, _ = sc.collide(ctx, db, torch.from_numpy(poses).cuda())
        work = sc.collide_last_tri_work(ctx)
        _, omd, _ = oracle.collide(b, poses)
        assert np.max(np.abs(gmd.cpu().numpy() - omd)) <= 1e-6
        assert 0 < work <= 3 * len(pts)


def test_mesh_arrays_validated(sc, ctx):
    """A batch that counts triangles but passes no triangle array is refused."""
    b = synth.meshes(seed=1, n_templates=2, cand_per_template=2)
    db = sc.DeviceBatch(b)
    db.c.tri = None
    with pytest.raises(sc.SceniError):
        sc.collide(ctx, db, db.new_poses())
    ctx.synchronize()


def test_triangle_limit_latches_device_code_9(sc, ctx):
    """A template with more than 65,536 triangles: the collision kernel
    latches device code 9 for its candidates and reports them as band."""
    n = 65537
    tri = np.zeros((n, 12), np.float32)
    tri[:, 0:3] = [5.0, 5.0, 5.0]
    tri[:, 4:7] = [5.1, 5.0, 5.0]
    tri[:, 8:11] = [5.0, 5.1, 5.0]
    b = tiny_batch([[(0.0, 0.0, 0.0, 0.01)]], n_cand=2)
    b.tmpl_tri_off, b.tri = np.array([0, n], np.int32), tri
    db = sc.DeviceBatch(b)
    _, _, band = sc.collide(ctx, db, db.new_poses())
    with pytest.raises(sc.SceniError) as ei:
        ctx.synchronize()
    assert "device error code 9" in str(ei.value)
    assert band.cpu().numpy().all()
    ctx.synchronize()
