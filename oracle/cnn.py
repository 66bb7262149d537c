"""Oracle of the learned displacement predictor (row a-L): plain float64 numpy.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and the CPU
legs of bench.py, never by the product path.

The paper predicts nothing: its level-0 displacements come from the SSD search of
Sec. 2.2. Row a-L replaces that search by a small convolutional network that
reads the normalized reference and the source pre-warped by the level-1
homography at quarter resolution and outputs one residual displacement per
32x32 tile (the plain search's displacement is its training label). This module
is the reference those kernels are checked against: a direct, unoptimized
statement of the network, its loss, its gradients and its optimizer step.

Network: a fixed feature stage, then learned layers. Features of a quarter-resolution
pixel p with inputs a = x[..., 0] (reference) and b = x[..., 1] (pre-warped source):
  a(p), b(p), and -(a(p) - b(p + o))^2 for the 25 offsets o = (u, v) in [-2, 2]^2
  (row-major in v then u; b = 0 outside the image)
-- a local SSD cost volume over +-8 full-resolution pixels, 27 channels. Learned
layers (in order), 3x3 convolutions with zero padding 1,
  c0: 27 -> 16 stride 1, c1: 16 -> 16 stride 1,
  c2: 16 -> 32 stride 2, c3: 32 -> 32 stride 1,
  c4: 32 -> 48 stride 2, c5: 48 -> 48 stride 1,
  c6: 48 -> 64 stride 2, c7: 64 -> 64 stride 1,
each followed by ReLU, then a 1x1 head h: 64 -> 2 without activation. A stride-2
output pixel (i, j) reads input pixels (2i + ky - 1, 2j + kx - 1), ky, kx in 0..2.
Tensors are NHWC. Parameters are one flat float32 vector: for every layer in
order, W[cout][ky][kx][cin] then b[cout] (the head as W[2][1][1][64], b[2]).

bf16=True rounds the values the CUDA path stores in bfloat16 (the input, the
features, the weights, every post-ReLU activation) to the nearest bfloat16, ties to even,
and keeps everything else in float64; bf16=False is the exact network (used for
the gradient pins).
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # (cin, cout, kernel, stride, relu)
    (27, 16, 3, 1, True), (16, 16, 3, 1, True),
    (16, 32, 3, 2, True), (32, 32, 3, 1, True),
    (32, 48, 3, 2, True), (48, 48, 3, 1, True),
    (48, 64, 3, 2, True), (64, 64, 3, 1, True),
    (64, 2, 1, 1, False),
]


def n_params(layers=LAYERS):
    return sum(co * k * k * ci + co for ci, co, k, s, r in layers)


def unpack(theta, layers=LAYERS):
    """Flat vector -> list of (W [cout, k, k, cin], b [cout]) as float64 views."""
    theta = np.asarray(theta, np.float64)
    out, o = [], 0
    for ci, co, k, s, r in layers:
        n = co * k * k * ci
        W = theta[o:o + n].reshape(co, k, k, ci)
        o += n
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    assert o == theta.size
    return out


def bf16_round(x):
    """Nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    r = np.where(np.isnan(f), u, r).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def init_params(seed, layers=LAYERS):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, head scaled by 0.1."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co, k, s, r) in enumerate(layers):
        std = np.sqrt(2.0 / (ci * k * k)) * (1.0 if r else 0.1)
        parts.append(rng.normal(0.0, std, co * k * k * ci))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def out_size(n, k, s):
    pad = k // 2
    return (n + 2 * pad - k) // s + 1


def conv_forward(x, W, b, stride):
    """Direct convolution: y[n, i, j, co] = b[co] + sum W[co, ky, kx, ci] x[n, s i + ky - p,
    s j + kx - p, ci] over taps inside the image (zero padding p = k // 2)."""
    n, h, w, ci = x.shape
    co, k, _, _ = W.shape
    p = k // 2
    ho, wo = out_size(h, k, stride), out_size(w, k, stride)
    xp = np.zeros((n, h + 2 * p, w + 2 * p, ci))
    xp[:, p:p + h, p:p + w, :] = x
    y = np.empty((n, ho, wo, co))
    y[...] = b
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, ky:ky + stride * (ho - 1) + 1:stride, kx:kx + stride * (wo - 1) + 1:stride, :]
            y += np.einsum("nhwc,oc->nhwo", patch, W[:, ky, kx, :])
    return y


def conv_backward(x, W, dy, stride):
    """Gradients of conv_forward: (dx, dW, db)."""
    n, h, w, ci = x.shape
    co, k, _, _ = W.shape
    p = k // 2
    ho, wo = dy.shape[1], dy.shape[2]
    xp = np.zeros((n, h + 2 * p, w + 2 * p, ci))
    xp[:, p:p + h, p:p + w, :] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(k):
        for kx in range(k):
            sl = (slice(None), slice(ky, ky + stride * (ho - 1) + 1, stride),
                  slice(kx, kx + stride * (wo - 1) + 1, stride), slice(None))
            dW[:, ky, kx, :] = np.einsum("nhwo,nhwc->oc", dy, xp[sl])
            dxp[sl] += np.einsum("nhwo,oc->nhwc", dy, W[:, ky, kx, :])
    db = dy.sum(axis=(0, 1, 2))
    return dxp[:, p:p + h, p:p + w, :], dW, db


CORR = 2  # offsets of the cost volume: [-CORR, CORR]^2


def features(x):
    """x [n, h, w, 2] -> [n, h, w, 2 + (2 CORR + 1)^2]: a, b, -(a(p) - b(p + o))^2."""
    n, h, w, _ = x.shape
    a, b = x[..., 0], x[..., 1]
    bp = np.zeros((n, h + 2 * CORR, w + 2 * CORR))
    bp[:, CORR:CORR + h, CORR:CORR + w] = b
    out = [a, b]
    for v in range(-CORR, CORR + 1):
        for u in range(-CORR, CORR + 1):
            d = a - bp[:, CORR + v:CORR + v + h, CORR + u:CORR + u + w]
            out.append(-(d * d))
    return np.stack(out, -1)


def forward(theta, x, bf16=False, layers=LAYERS, feature_stage=True, perturb=None):
    """x [n, h, w, 2] -> (out [n, h/8, w/8, 2] (ceil at each stride), cache for backward).
    feature_stage=False feeds x straight to the first layer (used by the gradient pins).
    perturb (tests only): a function applied to every layer's pre-activation, used to
    measure how far the bfloat16 chain moves under accumulation-sized noise."""
    params = unpack(theta, layers)
    if bf16:
        params = [(bf16_round(W), np.asarray(b, np.float32).astype(np.float64)) for W, b in params]
        x = bf16_round(x)
    x = np.asarray(x, np.float64)
    if feature_stage:
        x = features(x)
        if bf16:
            x = bf16_round(x)
    acts = [x]
    for (W, b), (ci, co, k, s, r) in zip(params, layers):
        z = conv_forward(acts[-1], W, b, s)
        if perturb is not None:
            z = perturb(z)
        if r:
            z = np.maximum(z, 0.0)
            if bf16:
                z = bf16_round(z)
        acts.append(z)
    return acts[-1], (params, acts)


def loss_and_grad_out(out, label, valid):
    """Mean squared error over valid cells: L = sum_valid |out - label|^2 / max(n_valid, 1);
    returns (L, dL/dout)."""
    v = np.asarray(valid, np.float64)[..., None]
    nv = max(float(v.sum()), 1.0)
    d = (out - label) * v
    return float((d * d).sum() / nv), 2.0 * d / nv


def backward(cache, dout, bf16=False, layers=LAYERS):
    """Flat gradient of the loss w.r.t. theta (float64), given dL/dout. bf16=True rounds
    each layer's output gradient (after the ReLU mask) to bfloat16, where the CUDA path
    stores it; the cache of a bf16 forward already holds bfloat16 weights and
    activations."""
    params, acts = cache
    grads = [None] * len(layers)
    g = dout
    for i in range(len(layers) - 1, -1, -1):
        ci, co, k, s, r = layers[i]
        W, b = params[i]
        if r:
            g = g * (acts[i + 1] > 0)
        if bf16:
            g = bf16_round(g)
        dx, dW, db = conv_backward(acts[i], W, g, s)
        grads[i] = (dW, db)
        g = dx
    return np.concatenate([np.concatenate([dW.reshape(-1), db]) for dW, db in grads])


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction at step t >= 1:
    m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
    theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
