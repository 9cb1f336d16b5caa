"""4D reachability map (RM4D-style, Sec. IV-E) through the C ABI against the
oracle: the cell of every target, the per-cell counts and the scores are
integers, so they must agree bit for bit; threshold tuning agrees exactly;
built from the IK kernel's own labels the map reaches its recall target."""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import synth
from oracle import rmap

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


def mixed_targets(seed, n):
    """Random orientations, top-down grasps with random yaw (the vertical
    approach case), a band of targets near cell edges, some outside the grid
    and a few degenerate rows."""
    rng = np.random.default_rng(seed)
    k = n // 3
    R = Rotation.random(k, random_state=rng).as_matrix().reshape(k, 9)
    p = rng.uniform([-1.6, -1.6, -1.3], [1.6, 1.6, 1.7], (k, 3))
    a = np.concatenate([R, p], 1)
    yaw = rng.uniform(0, 2 * math.pi, n - k)
    c, s = np.cos(yaw), np.sin(yaw)
    z0, z1 = np.zeros_like(c), np.ones_like(c)
    Rt = np.stack([c, s, z0, s, -c, z0, z0, z0, -z1], 1)
    pt = rng.uniform([-1.5, -1.5, -1.2], [1.5, 1.5, 1.6], (n - k, 3))
    pt[: (n - k) // 4, 0] = np.round(pt[: (n - k) // 4, 0] / 0.04375) * 0.04375  # on x* bin edges
    b = np.concatenate([Rt, pt], 1)
    t = np.concatenate([a, b]).astype(np.float32)
    t[:8] = 0.0
    t[8:12] = np.nan
    return t


@pytest.mark.parametrize("params", [(64, 16, 64, -1.1, 1.5, 1.4), (7, 3, 13, -0.3, 0.9, 0.77), (1, 1, 1, -2.0, 2.0, 2.0)])
def test_counts_and_scores_bit_identical(sc, ctx, params):
    t = mixed_targets(1, 60000)
    y = (np.random.default_rng(2).uniform(size=len(t)) < 0.45).astype(np.uint8)
    m = sc.ReachMap(ctx, params)
    assert m.cells == rmap.n_cells(params)
    tt, yy = torch.from_numpy(t).cuda(), torch.from_numpy(y).cuda()
    m.build(tt[:25000], yy[:25000])
    m.build(tt[25000:], yy[25000:])  # two builds add up to one
    got = m.counts()
    ref = rmap.build(params, t, y)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]
    s = m.query(tt).cpu().numpy()
    assert np.array_equal(s, rmap.score(params, ref, t))
    m.close()


def test_threshold_tuning_matches_oracle(sc, ctx):
    params = (32, 8, 32, -1.1, 1.5, 1.4)
    t = mixed_targets(3, 30000)
    y = (np.random.default_rng(4).uniform(size=len(t)) < 0.3).astype(np.uint8)
    tt, yy = torch.from_numpy(t).cuda(), torch.from_numpy(y).cuda()
    m = sc.ReachMap(ctx, params)
    m.build(tt[:20000], yy[:20000])
    ref_counts = rmap.build(params, t[:20000], y[:20000])
    for r in (0.5, 0.9, 0.99, 1.0):
        tau, rec, pr = m.tune_threshold(tt[20000:], yy[20000:], r)
        s = rmap.score(params, ref_counts, t[20000:])
        otau, orec, opr = rmap.tune(s, y[20000:], r)
        assert tau == otau and rec == pytest.approx(orec, abs=1e-6) and pr == pytest.approx(opr, abs=1e-6)
    m.close()


def test_empty_and_invalid(sc, ctx):
    m = sc.ReachMap(ctx, (4, 2, 4, 0.0, 1.0, 1.0))
    e = torch.empty((0, 12), dtype=torch.float32, device="cuda")
    m.build(e, torch.empty(0, dtype=torch.uint8, device="cuda"))
    assert m.query(e).numel() == 0
    assert m.counts().sum() == 0
    m.close()
    for bad in [(0, 1, 1, 0.0, 1.0, 1.0), (8, 8, 2048, 0.0, 1.0, 1.0), (4, 4, 4, 1.0, 1.0, 1.0),
                (4, 4, 4, 0.0, 1.0, 0.0), (4, 4, 4, 0.0, float("nan"), 1.0)]:
        with pytest.raises(sc.SceniError) as ei:
            sc.ReachMap(ctx, bad)
        assert ei.value.status == 1


def test_map_from_ik_labels_reaches_recall(sc, ctx):
    """Built from the IK kernel's labels of top-down grasps over the workload's
    region, the map tuned on held-out targets keeps >= 99% of the reachable
    ones and rejects a real share of the rest."""
    arm = sc.make_arm(*synth.arm_arrays())
    box = ((-0.2, 2.2), (-1.3, 1.3), (0.0, 0.8))
    tr = torch.from_numpy(synth.topdown_targets(seed=11, n=262144, box=box)).cuda()
    ho = torch.from_numpy(synth.topdown_targets(seed=12, n=65536, box=box)).cuda()
    ytr, _, _ = sc.ik_reach(ctx, arm, sc.ik_params(seed=11), tr)
    yho, _, _ = sc.ik_reach(ctx, arm, sc.ik_params(seed=12), ho)
    m = sc.ReachMap(ctx, (32, 16, 32, -1.1, 1.5, 1.4))  # ~9 cm cells: about 25 labels per visited cell
    m.build(tr, ytr)
    tau, rec, pr = m.tune_threshold(ho, yho, 0.99)
    assert rec >= 0.99 and tau >= 1
    assert pr < 0.6, pr  # reachable share of these targets is ~0.14
    assert pr >= yho.float().mean().item() * rec - 1e-6
    m.close()
