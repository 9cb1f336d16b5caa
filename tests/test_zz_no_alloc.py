"""sc_collide_noalloc: the collision check for callers that cannot allocate.

Callers whose device memory is owned by a framework pool, or that run a
per-frame loop where cudaMalloc would stall the device, or that keep no
library context, use this entry point: it takes no sc_ctx and keeps its
scratch in a fixed array inside the library. These tests call it through the
C ABI and check that it returns what sc_collide returns for the same inputs,
on two calls in a row (the second call must not see the first call's
scratch). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL_DIST = 1e-5  # the distance tolerance of the parity tests


@pytest.fixture(scope="module")
def sc():
    import paper_2512_16896_b300 as sc
    from paper_2512_16896_b300 import build
    build.build()
    return sc


def _noalloc(sc, db, poses, active=None, first_new=0):
    L = sc.lib()
    n = db.n_cand if active is None else active.numel()
    col = torch.empty(n, dtype=torch.uint8, device="cuda")
    md = torch.empty(n, dtype=torch.float32, device="cuda")
    band = torch.empty(n, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.sc_collide_noalloc(stream, ctypes.byref(db.c), ctypes.c_void_p(poses.data_ptr()),
                              None if active is None else ctypes.c_void_p(active.data_ptr()), n, first_new,
                              ctypes.c_void_p(col.data_ptr()), ctypes.c_void_p(md.data_ptr()),
                              ctypes.c_void_p(band.data_ptr()))
    assert st == 0, L.sc_last_error()
    return col, md, band


def _same(a, b):
    ca, ma, ba = (x.cpu().numpy() for x in a)
    cb, mb, bb = (x.cpu().numpy() for x in b)
    assert np.array_equal(ca, cb) and np.array_equal(ba, bb)
    assert np.max(np.abs(ma.astype(np.float64) - mb.astype(np.float64)), initial=0.0) <= TOL_DIST


def test_noalloc_matches_collide_twice(sc):
    ctx = sc.Context()
    try:
        first = synth.shelf(seed=21, n_cand=700, n_obj=12, n_sph=24, n_obb=6)
        second = synth.ragged(seed=22, n_templates=40, cand_per_template=9)
        for b, seed, first_new in ((first, 1, 0), (second, 2, 3)):
            db = sc.DeviceBatch(b)
            poses = torch.from_numpy(synth.random_poses(b, seed=seed, spread=0.5)).cuda()
            order = torch.from_numpy(sc.order_by_work(b)).cuda()
            ref = sc.collide(ctx, db, poses, active=order, first_new=first_new)
            got = _noalloc(sc, db, poses, active=order, first_new=first_new)
            torch.cuda.synchronize()
            _same(ref, got)
        # and once more on the first batch, all candidates, no list
        db = sc.DeviceBatch(first)
        poses = torch.from_numpy(synth.random_poses(first, seed=3)).cuda()
        ref = sc.collide(ctx, db, poses)
        got = _noalloc(sc, db, poses)
        torch.cuda.synchronize()
        _same(ref, got)
        ctx.synchronize()
    finally:
        ctx.close()


def test_noalloc_rejects_oversized_list(sc):
    """More candidates than the per-call limit (the 32-bit work counter): refused on the host."""
    L = sc.lib()
    b = synth.tabletop(seed=0, n_cand=4)
    db = sc.DeviceBatch(b)
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = torch.zeros(8, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(out.data_ptr())
    st = L.sc_collide_noalloc(None, ctypes.byref(db.c), p, ctypes.c_void_p(dummy.data_ptr()), (1 << 30) + 1, 0, p, p, p)
    assert st == 1
    assert b"limit" in L.sc_last_error()


def test_noalloc_marks_a_malformed_part_box(sc):
    """A world box naming a part its template lacks: there is no status word
    here, so the candidate itself must say it has no verdict (NaN, band 1,
    not colliding), and the next call on well-formed input is unaffected."""
    from scenes import tiny_batch
    part = [[1.0, 0.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.2, 0.2, 0.0, 0.0]]
    bad = tiny_batch([[(0, 0, 0, 0.01)]], obbs=[[0.5, 0, 0, 0, 0, 0, 0, 1, 0.1, 0.1, 0.1, 0]], n_cand=3,
                     parts=part, obb_part=[3])
    db = sc.DeviceBatch(bad)
    col, md, band = _noalloc(sc, db, db.new_poses())
    torch.cuda.synchronize()
    assert np.all(np.isnan(md.cpu().numpy())) and np.all(band.cpu().numpy() == 1) and np.all(col.cpu().numpy() == 0)
    good = tiny_batch([[(0, 0, 0, 0.01)]], obbs=[[0.5, 0, 0, 0, 0, 0, 0, 1, 0.1, 0.1, 0.1, 0]], n_cand=3,
                      parts=part, obb_part=[0])
    dg = sc.DeviceBatch(good)
    col, md, band = _noalloc(sc, dg, dg.new_poses())
    torch.cuda.synchronize()
    assert np.all(np.isfinite(md.cpu().numpy())) and np.all(band.cpu().numpy() == 0)
