"""FP64 CPU oracle of the learned warm-start network (a small 3-D U-Net) and its gradients.

TEST INFRASTRUCTURE ONLY: used by tests to check the CUDA network kernels; never imported by the
product path.  Plain numpy float64, written from the definitions (3-D cross-correlation with
periodic padding, ReLU, 2x2x2 average pooling, nearest-neighbour 2x upsampling, channel concat, mean
squared error) with explicit loops over the 27 taps; the backward pass is the chain rule of the same
definitions.  The test suite pins it against central finite differences.

Tensors are channels-last: x[z0, z1, z2, c] on a periodic n^3 grid.  A 3x3x3 convolution with
weights w[tap, cin, cout] (tap = (dx+1)*9 + (dy+1)*3 + (dz+1)) and bias b[cout] computes
    y[v, co] = b[co] + sum_tap sum_ci x[v + d(tap), ci] w[tap, ci, co]     (indices mod n).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]

# (name, cin, cout) of the network, in order.  Input channels: smoothed delta, the three
# line-of-sight components, and the radial displacement of the Eq. approx2 start; the head adds its
# output to that last input channel, so the network learns the correction to the start.
def layer_specs(c1: int = 16, cin: int = 5):
    c2, c3 = 2 * c1, 4 * c1
    return [
        ("enc1a", cin, c1), ("enc1b", c1, c1),
        ("enc2a", c1, c2), ("enc2b", c2, c2),
        ("bota", c2, c3), ("botb", c3, c3),
        ("dec2a", c3 + c2, c2), ("dec2b", c2, c2),
        ("dec1a", c2 + c1, c1), ("dec1b", c1, c1),
        ("head", c1, 1),
    ]


def init_params(seed: int, c1: int = 16, cin: int = 5):
    """He-normal weights (the head starts at zero so the network starts as the identity correction)."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co in layer_specs(c1, cin):
        if name == "head":
            params[name] = (np.zeros((1, ci, co)), np.zeros(co))
        else:
            std = np.sqrt(2.0 / (27 * ci))
            params[name] = (rng.standard_normal((27, ci, co)) * std, np.zeros(co))
    return params


def conv3(x, w, b):
    """Periodic 3x3x3 cross-correlation (or 1x1x1 when w has one tap)."""
    y = np.broadcast_to(b, x.shape[:3] + (w.shape[2],)).copy()
    taps = TAPS if w.shape[0] == 27 else [(0, 0, 0)]
    for t, (dx, dy, dz) in enumerate(taps):
        xs = np.roll(x, shift=(-dx, -dy, -dz), axis=(0, 1, 2))      # xs[v] = x[v + d]
        y += xs @ w[t]
    return y


def conv3_backward(x, w, gy):
    """Gradients of conv3 w.r.t. x, w, b given the output gradient gy."""
    taps = TAPS if w.shape[0] == 27 else [(0, 0, 0)]
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dx, dy, dz) in enumerate(taps):
        xs = np.roll(x, shift=(-dx, -dy, -dz), axis=(0, 1, 2))
        gw[t] = xs.reshape(-1, x.shape[3]).T @ gy.reshape(-1, gy.shape[3])
        gx += np.roll(gy @ w[t].T, shift=(dx, dy, dz), axis=(0, 1, 2))
    gb = gy.reshape(-1, gy.shape[3]).sum(0)
    return gx, gw, gb


def pool2(x):
    n = x.shape[0]
    return x.reshape(n // 2, 2, n // 2, 2, n // 2, 2, -1).mean(axis=(1, 3, 5))


def pool2_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, 0), 2, 1), 2, 2) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up2_backward(gy):
    n = gy.shape[0]
    return gy.reshape(n // 2, 2, n // 2, 2, n // 2, 2, -1).sum(axis=(1, 3, 5))


def forward(params, x):
    """Network output and the activations the backward pass needs."""
    a = {}
    h = x
    for name in ("enc1a", "enc1b"):
        a[name + ".in"] = h
        h = np.maximum(conv3(h, *params[name]), 0.0)
        a[name + ".out"] = h
    s1 = h
    h = pool2(s1)
    for name in ("enc2a", "enc2b"):
        a[name + ".in"] = h
        h = np.maximum(conv3(h, *params[name]), 0.0)
        a[name + ".out"] = h
    s2 = h
    h = pool2(s2)
    for name in ("bota", "botb"):
        a[name + ".in"] = h
        h = np.maximum(conv3(h, *params[name]), 0.0)
        a[name + ".out"] = h
    h = np.concatenate([up2(h), s2], axis=3)
    for name in ("dec2a", "dec2b"):
        a[name + ".in"] = h
        h = np.maximum(conv3(h, *params[name]), 0.0)
        a[name + ".out"] = h
    h = np.concatenate([up2(h), s1], axis=3)
    for name in ("dec1a", "dec1b"):
        a[name + ".in"] = h
        h = np.maximum(conv3(h, *params[name]), 0.0)
        a[name + ".out"] = h
    a["head.in"] = h
    y = conv3(h, *params["head"]) + x[..., -1:]
    return y, a


def loss(params, x, target):
    """Mean squared error over all voxels."""
    y, _ = forward(params, x)
    return float(((y - target) ** 2).mean())


def backward(params, x, target):
    """Loss and its gradients {name: (gw, gb)} by the chain rule."""
    y, a = forward(params, x)
    diff = y - target
    L = float((diff ** 2).mean())
    g = 2.0 * diff / diff.size
    grads = {}

    def conv_relu_back(name, gout):
        gout = gout * (a[name + ".out"] > 0)
        gx, gw, gb = conv3_backward(a[name + ".in"], params[name][0], gout)
        grads[name] = (gw, gb)
        return gx

    gx, gw, gb = conv3_backward(a["head.in"], params["head"][0], g)
    grads["head"] = (gw, gb)
    g = conv_relu_back("dec1b", gx)
    g = conv_relu_back("dec1a", g)
    c2 = params["dec2b"][0].shape[2]
    g_up, g_s1 = g[..., :c2], g[..., c2:]
    g = up2_backward(g_up)
    g = conv_relu_back("dec2b", g)
    g = conv_relu_back("dec2a", g)
    c3 = params["botb"][0].shape[2]
    g_up, g_s2 = g[..., :c3], g[..., c3:]
    g = up2_backward(g_up)
    g = conv_relu_back("botb", g)
    g = conv_relu_back("bota", g)
    g = pool2_backward(g) + g_s2
    g = conv_relu_back("enc2b", g)
    g = conv_relu_back("enc2a", g)
    g = pool2_backward(g) + g_s1
    g = conv_relu_back("enc1b", g)
    conv_relu_back("enc1a", g)
    return L, grads


def adamw(params, grads, state, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One decoupled-weight-decay Adam update (weights only decay; biases do not)."""
    out = {}
    for name, (w, b) in params.items():
        gw, gb = grads[name]
        mw, vw, mb, vb = state.get(name, (np.zeros_like(w), np.zeros_like(w), np.zeros_like(b), np.zeros_like(b)))
        mw = beta1 * mw + (1 - beta1) * gw
        vw = beta2 * vw + (1 - beta2) * gw * gw
        mb = beta1 * mb + (1 - beta1) * gb
        vb = beta2 * vb + (1 - beta2) * gb * gb
        c1, c2 = 1 - beta1 ** step, 1 - beta2 ** step
        w = w - lr * (mw / c1 / (np.sqrt(vw / c2) + eps) + wd * w)
        b = b - lr * (mb / c1 / (np.sqrt(vb / c2) + eps))
        out[name] = (w, b)
        state[name] = (mw, vw, mb, vb)
    return out
