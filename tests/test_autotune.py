"""The launch-shape autotuner: its cache key on the host, and on the GPU that
the shapes it picks compute exactly what the default shape computes (a launch
shape only changes how the work is spread over CTAs and warps)."""
import numpy as np
import pytest

import synth
from paper_2512_16896_b300 import autotune


def test_shape_key_is_stable_and_tells_shapes_apart():
    a = synth.ragged(seed=1, n_templates=32, cand_per_template=4)
    b = synth.ragged(seed=1, n_templates=32, cand_per_template=4)
    assert autotune.shape_key(a, 0) == autotune.shape_key(b, 0)
    assert autotune.shape_key(a, 0) != autotune.shape_key(a, 3)  # whole scene vs. re-check of later objects
    t = synth.tabletop(seed=0, n_cand=64)
    s = synth.shelf(seed=1, n_cand=64, n_obj=12, n_sph=24, n_obb=6)
    assert len({autotune.shape_key(x, 0) for x in (a, t, s)}) == 3
    ka = autotune.generate_key(a, 10, True, True)
    assert ka == autotune.generate_key(b, 10, True, True)
    assert len({ka, autotune.generate_key(a, 0, True, True), autotune.generate_key(a, 10, False, False),
                autotune.generate_key(a, 10, True, False)}) == 4


def test_search_spaces_are_launchable_shapes():
    for t, apl, seg, cps in autotune.DEFAULT_SPACE:
        assert apl in (1, 2, 4) and 128 <= t <= (512 if apl == 4 else 1024) and t % 32 == 0
        assert 8 <= seg <= 4096 and seg % 8 == 0 and 1 <= cps <= 8
    for t, apl, seg, cps in autotune.GENERATE_SPACE:  # the generation kernels take at most 256 threads
        assert apl in (1, 2, 4) and t in (128, 256) and 1 <= cps <= 8


@pytest.fixture(scope="module")
def gpu():
    import torch
    import paper_2512_16896_b300 as sc
    from paper_2512_16896_b300 import build
    build.build()
    ctx = sc.Context()
    yield sc, ctx, torch
    ctx.close()


@pytest.mark.gpu
def test_tuned_collision_shape_is_bit_identical(gpu):
    sc, ctx, torch = gpu
    b = synth.ragged(seed=31, n_templates=48, cand_per_template=8, obj_range=(2, 24))
    db = sc.DeviceBatch(b)
    poses = torch.from_numpy(synth.random_poses(b, seed=3, spread=0.5)).cuda()
    order = torch.from_numpy(sc.order_by_work(b)).cuda()
    space = [(256, 4, 256, 4), (128, 2, 128, 2), (512, 4, 512, 1)]
    best, entry = autotune.tune_collide(ctx, db, b, poses, order, space=space, use_cache=False)
    assert tuple(best)[:4] in space and best[4] == 0 and best[5] in (0, 1) and entry["sample"] == order.numel()
    ref = sc.collide(ctx, db, poses, active=order)
    got = sc.collide(ctx, db, poses, active=order, config=best)
    for x, y in zip(ref, got):
        assert torch.equal(x, y)


@pytest.mark.gpu
def test_tuned_generation_shape_is_bit_identical(gpu):
    sc, ctx, torch = gpu
    b = synth.ragged(seed=32, n_templates=24, cand_per_template=8, obj_range=(2, 12))
    db = sc.DeviceBatch(b)
    order = torch.from_numpy(sc.order_by_work(b)).cuda()
    arm = sc.make_arm(*synth.arm_arrays())
    ik = sc.ik_params(seed=5)
    space = [(256, 1, 256, 4), (128, 2, 256, 3), (128, 1, 256, 6)]
    best, entry = autotune.tune_generate(ctx, db, b, order, seed=5, arm=arm, ik=ik, space=space, use_cache=False)
    assert tuple(best) in space
    ref = [x.clone() for x in sc.generate(ctx, db, seed=5, order=order, arm=arm, ik=ik)]
    got = [x.clone() for x in sc.generate(ctx, db, seed=5, order=order, arm=arm, ik=ik, config=best)]
    ctx.synchronize()
    assert ref[1].sum().item() > 0
    for x, y in zip(ref, got):
        assert torch.equal(torch.nan_to_num(x, 7.0), torch.nan_to_num(y, 7.0))
