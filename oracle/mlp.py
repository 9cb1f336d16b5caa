"""FP64 oracle of the reachability surrogate (TEST INFRASTRUCTURE ONLY).

The paper answers "can the robot reach this pose?" with an RM4D map (Sec. IV-E).
This build answers it exactly with IK and puts a small learned filter in front
of the exact check: an MLP 9 -> 256 -> 256 -> 256 -> 1 with SiLU activations,
trained with binary cross-entropy on logits and Adam.

Definitions followed here (plain numpy; matmul is the only library step):
  features  x = (p, R[:,0], R[:,1])     position + 6D rotation (Zhou et al., CVPR 2019)
  standardise  x_hat = (x - mu) / sigma   (mu, sigma stored with the weights)
  a_l = W_l h_{l-1} + b_l,  h_l = SiLU(a_l) = a_l * sigmoid(a_l),  l = 1..3
  z   = W_4 h_3 + b_4                     (logit)
  BCE(z, y) = max(z, 0) - z y + log(1 + exp(-|z|)),  mean over the batch
  Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
        w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

Mixed precision of the GPU kernels, reproduced when bf16=True: the compute
copies of W_1..W_4 are the FP32 master weights rounded to bfloat16; x_hat and
every h_l are rounded to bfloat16; in the backward pass every dL/da_l is
rounded to bfloat16 before it enters a product; biases, pre-activations,
accumulations, gradients and Adam state stay in high precision.
Pinned by: bf16 rounding == torch's float32->bfloat16 conversion; backward
(bf16=False) == central finite differences of the FP64 loss; BCE(0) = ln 2;
Adam's first step from zero moments = -lr g / (|g| + eps').
"""
from __future__ import annotations

import numpy as np

WIDTHS = (9, 256, 256, 256, 1)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    The value is first rounded to float32 (the GPU holds it in float32 before
    converting), then its low 16 bits are rounded off with ties to even."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def features(targets: np.ndarray) -> np.ndarray:
    """[n,12] targets (R row-major, p) -> [n,9] features (p, first two columns of R)."""
    t = np.asarray(targets, np.float64).reshape(-1, 12)
    R = t[:, :9].reshape(-1, 3, 3)
    return np.concatenate([t[:, 9:12], R[:, :, 0], R[:, :, 1]], axis=1)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(a):
    return a * sigmoid(a)


def silu_grad(a):
    s = sigmoid(a)
    return s * (1.0 + a * (1.0 - s))


def bce_with_logits(z, y):
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    return np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))


class Params:
    """FP32 master parameters (stored as float64 copies of float32 values)."""

    def __init__(self, W, b, mu, sigma):
        self.W = [np.asarray(w, np.float64) for w in W]  # W[l]: [out, in]
        self.b = [np.asarray(v, np.float64) for v in b]
        self.mu = np.asarray(mu, np.float64)
        self.sigma = np.asarray(sigma, np.float64)


def forward(P: Params, targets, bf16=True):
    """Returns (logits [n], cache) with cache = (x_hat, [a_l], [h_l])."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    x = (features(targets) - P.mu) / P.sigma
    h = rnd(x)
    hs, As = [h], []
    for l in range(3):
        a = h @ rnd(P.W[l]).T + P.b[l]
        As.append(a)
        h = rnd(silu(a))
        hs.append(h)
    z = h @ rnd(P.W[3]).T + P.b[3]
    return z[:, 0], (hs, As)


def loss(P: Params, targets, y, bf16=True):
    z, _ = forward(P, targets, bf16)
    return float(np.mean(bce_with_logits(z, y)))


def backward(P: Params, targets, y, bf16=True):
    """Mean-BCE loss and its gradients (dW list, db list)."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    z, (hs, As) = forward(P, targets, bf16)
    n = len(z)
    y = np.asarray(y, np.float64)
    L = float(np.mean(bce_with_logits(z, y)))
    dz = (sigmoid(z) - y)[:, None] / n  # dL/dz, [n,1]
    dW = [None] * 4
    db = [None] * 4
    dW[3] = dz.T @ hs[3]
    db[3] = dz.sum(axis=0)
    g = rnd(dz) @ rnd(P.W[3])  # dL/dh_3
    for l in (2, 1, 0):
        da = rnd(g * silu_grad(As[l]))
        dW[l] = da.T @ hs[l]
        db[l] = da.sum(axis=0)
        if l > 0:
            g = da @ rnd(P.W[l])
    return L, dW, db


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = 1-based step). Returns new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(rng: np.random.Generator, mu=None, sigma=None) -> Params:
    """U(+-1/sqrt(fan_in)) weights and biases (float32 values)."""
    W, b = [], []
    for l in range(4):
        fi, fo = WIDTHS[l], WIDTHS[l + 1]
        k = 1.0 / np.sqrt(fi)
        W.append(rng.uniform(-k, k, size=(fo, fi)).astype(np.float32))
        b.append(rng.uniform(-k, k, size=(fo,)).astype(np.float32))
    mu = np.zeros(9) if mu is None else mu
    sigma = np.ones(9) if sigma is None else sigma
    return Params(W, b, mu, sigma)
