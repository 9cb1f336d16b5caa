"""Surrogate MLP kernels (BF16 tensor cores, FP32 accumulation) against the
FP64 oracle that reproduces the same bf16 rounding points, through the C ABI.

Tolerances: logits within 2e-2 x max(1, |z|max) (mean within 2e-3); every
gradient tensor within 2e-2 x its largest reference entry with cosine
>= 0.999; an Adam step within 1e-6. Training uses labels from the project's
own IK kernel; the tuned gate keeps recall >= 0.99 on held-out targets.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

H = 256


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


def pack(P):
    return np.concatenate([P.W[0].ravel(), P.b[0], P.W[1].ravel(), P.b[1], P.W[2].ravel(), P.b[2], P.W[3].ravel(),
                           P.b[3]]).astype(np.float32)


def unpack(flat):
    o, out = 0, []
    for shape in [(H, 9), (H,), (H, H), (H,), (H, H), (H,), (1, H), (1,)]:
        n = int(np.prod(shape))
        out.append(flat[o:o + n].reshape(shape))
        o += n
    return out


def random_net(seed):
    rng = np.random.default_rng(seed)
    P = omlp.init_params(rng, mu=rng.normal(size=9) * 0.2, sigma=rng.uniform(0.3, 1.5, 9))
    # round the stored values to float32 (the GPU masters are float32)
    P.W = [w.astype(np.float32).astype(np.float64) for w in P.W]
    P.b = [b.astype(np.float32).astype(np.float64) for b in P.b]
    P.mu = P.mu.astype(np.float32).astype(np.float64)
    P.sigma = P.sigma.astype(np.float32).astype(np.float64)
    return P


# 1 row; a ragged tail past 128-row tiles; more tiles than CTAs (each CTA
# takes several tiles and reloads the layer weights between them)
@pytest.mark.parametrize("n", [1, 4099, 2 * 148 * 128 + 77])
def test_forward_matches_oracle(sc, ctx, n):
    P = random_net(1)
    net = sc.Surrogate(ctx, seed=0)
    net.set(pack(P), P.mu, P.sigma, 0.0)
    tg = synth.topdown_targets(seed=11, n=n)
    z = net.infer(torch.from_numpy(tg).cuda()).cpu().numpy().astype(np.float64)
    ctx.synchronize()  # raises if a bounded device wait gave up
    zr, _ = omlp.forward(P, tg, bf16=True)
    scale = max(1.0, np.abs(zr).max())
    assert np.abs(z - zr).max() <= 2e-2 * scale, np.abs(z - zr).max()
    assert np.abs(z - zr).mean() <= 2e-3 * scale
    net.close()


# one 4096-row batch (32 tiles); a ragged batch (a partial tile and a
# partial 64-row chunk of the weight-gradient reduction); more tiles than the
# GPU holds at once; and small batches whose weight-gradient clusters have
# 1, 2 and 5 CTAs (a split count that is no power of two; 128 / S rows of the
# cross-split reduction per CTA, in several blocks for S <= 2)
@pytest.mark.parametrize("n", [4096, 1000, 2 * 148 * 128 + 77, 1, 100, 300])
def test_gradients_match_oracle(sc, ctx, n):
    P = random_net(2)
    net = sc.Surrogate(ctx, seed=0)
    net.set(pack(P), P.mu, P.sigma, 0.0)
    tg = synth.topdown_targets(seed=12, n=n)
    y = (np.random.default_rng(3).uniform(size=n) < 0.5).astype(np.uint8)
    g, loss = net.grads(torch.from_numpy(tg).cuda(), torch.from_numpy(y).cuda())
    g = g.cpu().numpy().astype(np.float64)
    L, dW, db = omlp.backward(P, tg, y.astype(np.float64), bf16=True)
    assert loss == pytest.approx(L, rel=1e-3)
    ref = [dW[0], db[0], dW[1], db[1], dW[2], db[2], dW[3], db[3]]
    for got, want, name in zip(unpack(g), ref, ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]):
        want = np.asarray(want).reshape(got.shape)
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 2e-2 * scale, (name, np.abs(got - want).max(), scale)
        cos = float(np.dot(got.ravel(), want.ravel()) / (np.linalg.norm(got) * np.linalg.norm(want) + 1e-30))
        assert cos >= 0.999, (name, cos)
    net.close()


# The fused training step (the weight-gradient kernel applies Adam to each
# gradient it writes) leaves the same bits as the gradient call followed by
# the Adam call, over two steps (bias corrections of t = 1 and 2); one full
# batch and a ragged one.
@pytest.mark.parametrize("n", [4096, 1000])
def test_fused_train_step_equals_gradients_then_adam(sc, ctx, n):
    P = random_net(5)
    a, b = sc.Surrogate(ctx, seed=0), sc.Surrogate(ctx, seed=0)
    for net in (a, b):
        net.set(pack(P), P.mu, P.sigma, 0.0)
    tg = torch.from_numpy(synth.topdown_targets(seed=13, n=n)).cuda()
    y = torch.from_numpy((np.random.default_rng(6).uniform(size=n) < 0.5).astype(np.uint8)).cuda()
    tp = sc.train_params(lr=1e-3)
    for _ in range(2):
        _, la = a.grads(tg, y)
        a.adam_step(None, tp)  # the gradients the last call left on the device
        lb = b.train_step(tg, y, tp)
        assert la == lb
    pa, pb = a.get()[0], b.get()[0]
    assert np.array_equal(pa, pb), np.abs(pa - pb).max()
    assert not np.array_equal(pa, pack(P))
    assert torch.equal(a.infer(tg), b.infer(tg))  # the bf16 weight copies agree too
    a.close()
    b.close()


def test_adam_step_matches_formula(sc, ctx):
    P = random_net(3)
    net = sc.Surrogate(ctx, seed=0)
    w0 = pack(P)
    net.set(w0, P.mu, P.sigma, 0.0)
    rng = np.random.default_rng(4)
    grads = (rng.normal(size=w0.size) * 10.0 ** rng.integers(-6, 0, w0.size)).astype(np.float32)
    tp = sc.train_params(lr=1e-3)
    net.adam_step(torch.from_numpy(grads).cuda(), tp)
    net.adam_step(torch.from_numpy(grads * 0.5).cuda(), tp)
    w2 = net.get()[0].astype(np.float64)
    w, m, v = w0.astype(np.float64), np.zeros(w0.size), np.zeros(w0.size)
    w, m, v = omlp.adam_step(w, grads.astype(np.float64), m, v, 1)
    w, m, v = omlp.adam_step(w, 0.5 * grads.astype(np.float64), m, v, 2)
    assert np.abs(w2 - w).max() <= 1e-6
    net.close()


def test_training_on_ik_labels_and_gate_recall(sc, ctx, tmp_path):
    arm = sc.make_arm(*synth.arm_arrays())
    tr = torch.from_numpy(synth.topdown_targets(seed=4, n=131072)).cuda()
    ho = torch.from_numpy(synth.topdown_targets(seed=5, n=32768)).cuda()
    ytr, _, _ = sc.ik_reach(ctx, arm, sc.ik_params(seed=4), tr)
    yho, _, _ = sc.ik_reach(ctx, arm, sc.ik_params(seed=5), ho)
    net = sc.Surrogate(ctx, seed=7)
    z0 = net.infer(ho)
    loss = net.train(tr, ytr, sc.train_params(epochs=6, batch=4096, seed=4))
    assert loss[-1] < 0.45 and loss[-1] < loss[0], loss
    tau, rec, pass_rate = net.tune_threshold(ho, yho, 0.99)
    assert rec >= 0.99
    assert pass_rate < 0.9  # the gate rejects a real share of targets
    # labels of the held-out set: the gate's false negatives are at most 1%
    z = net.infer(ho)
    pos = yho.bool()
    assert ((z >= tau) & pos).sum().item() >= 0.99 * pos.sum().item()
    # checkpoint round trip
    path = str(tmp_path / "gate.bin")
    net.save(path)
    net2 = sc.Surrogate.load(ctx, path)
    assert torch.equal(net2.infer(ho), z)
    assert net2.get()[3] == pytest.approx(tau)
    assert not torch.equal(z0, z)
    net.close()
    net2.close()
