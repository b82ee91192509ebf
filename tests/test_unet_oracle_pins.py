"""Pins of the FP64 U-Net oracle: convolution against a brute-force loop, gradients against central
finite differences, pooling/upsampling adjointness."""
import numpy as np
import pytest

from oracle import unet_oracle as U


def brute_conv(x, w, b):
    n = x.shape[0]
    y = np.zeros(x.shape[:3] + (w.shape[2],))
    for i in range(n):
        for j in range(n):
            for k in range(n):
                acc = b.copy()
                for t, (dx, dy, dz) in enumerate(U.TAPS):
                    acc = acc + x[(i + dx) % n, (j + dy) % n, (k + dz) % n] @ w[t]
                y[i, j, k] = acc
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((4, 4, 4, 3))
    w = rng.standard_normal((27, 3, 5))
    b = rng.standard_normal(5)
    assert np.abs(U.conv3(x, w, b) - brute_conv(x, w, b)).max() < 1e-12


def test_conv_backward_adjoint():
    """<conv(x), gy> = <x, conv_backward(gy)> (linear part) and weight gradient by definition."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 4, 4, 3))
    w = rng.standard_normal((27, 3, 2))
    gy = rng.standard_normal((4, 4, 4, 2))
    gx, gw, gb = U.conv3_backward(x, w, gy)
    assert np.isclose((U.conv3(x, w, np.zeros(2)) * gy).sum(), (x * gx).sum(), rtol=1e-12)
    eps = 1e-6
    for (t, ci, co) in [(0, 0, 0), (13, 2, 1), (26, 1, 0)]:
        wp = w.copy(); wp[t, ci, co] += eps
        wm = w.copy(); wm[t, ci, co] -= eps
        fd = ((U.conv3(x, wp, np.zeros(2)) - U.conv3(x, wm, np.zeros(2))) * gy).sum() / (2 * eps)
        assert np.isclose(fd, gw[t, ci, co], rtol=1e-6)
    assert np.allclose(gb, gy.reshape(-1, 2).sum(0))


def test_pool_up_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 4, 4, 3))
    y = rng.standard_normal((2, 2, 2, 3))
    assert np.isclose((U.pool2(x) * y).sum(), (x * U.pool2_backward(y)).sum(), rtol=1e-12)
    assert np.isclose((U.up2(y) * x).sum(), (y * U.up2_backward(x)).sum(), rtol=1e-12)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    n, c1 = 8, 2
    params = U.init_params(4, c1=c1, cin=5)
    # a non-zero head so every layer receives gradient
    params["head"] = (rng.standard_normal((1, c1, 1)) * 0.5, np.array([0.1]))
    for k in params:
        w, b = params[k]
        params[k] = (w, b + 0.05 * rng.standard_normal(b.shape))
    x = rng.standard_normal((n, n, n, 5))
    target = rng.standard_normal((n, n, n, 1))
    L, grads = U.backward(params, x, target)
    eps = 1e-6
    for name in ("enc1a", "enc2b", "bota", "dec2a", "dec1b", "head"):
        w, b = params[name]
        idx = tuple(rng.integers(0, s) for s in w.shape)
        for which in ("w", "b"):
            p_plus = dict(params)
            p_minus = dict(params)
            if which == "w":
                wp = w.copy(); wp[idx] += eps
                wm = w.copy(); wm[idx] -= eps
                p_plus[name], p_minus[name] = (wp, b), (wm, b)
                g = grads[name][0][idx]
            else:
                j = rng.integers(0, b.shape[0])
                bp = b.copy(); bp[j] += eps
                bm = b.copy(); bm[j] -= eps
                p_plus[name], p_minus[name] = (w, bp), (w, bm)
                g = grads[name][1][j]
            fd = (U.loss(p_plus, x, target) - U.loss(p_minus, x, target)) / (2 * eps)
            assert fd == pytest.approx(g, rel=1e-5, abs=1e-10), (name, which)


def test_zero_head_returns_the_start():
    """With the initial (zero) head the network returns its last input channel: the start estimate."""
    params = U.init_params(5)
    x = np.random.default_rng(6).standard_normal((8, 8, 8, 5))
    y, _ = U.forward(params, x)
    assert np.array_equal(y, x[..., -1:])


def _one_layer(seed):
    rng = np.random.default_rng(seed)
    return {"l": (rng.standard_normal((27, 2, 3)), rng.standard_normal(3))}


def test_adamw_first_step_is_a_unit_sign_step_plus_decay():
    """AdamW (Loshchilov & Hutter, decoupled decay): from zero moments the bias-corrected first and
    second moments are g and g^2, so the first step moves each weight by lr (g / (|g| + eps) + wd w)
    and each bias by lr g / (|g| + eps) (biases do not decay)."""
    p = _one_layer(1)
    g = _one_layer(2)
    lr, wd, eps = 3e-3, 1e-2, 1e-8
    out = U.adamw(p, g, {}, lr, 1, eps=eps, wd=wd)
    (w0, b0), (gw, gb), (w1, b1) = p["l"], g["l"], out["l"]
    assert np.abs(w1 - (w0 - lr * (gw / (np.abs(gw) + eps) + wd * w0))).max() < 1e-14
    assert np.abs(b1 - (b0 - lr * gb / (np.abs(gb) + eps))).max() < 1e-14


def test_adamw_constant_gradient_and_pure_decay():
    """A constant gradient keeps the bias-corrected moments exactly g and g^2 at every step, so T
    steps without decay move by T lr g / (|g| + eps); a zero gradient leaves only the decoupled decay,
    w_T = w_0 (1 - lr wd)^T, and the biases fixed."""
    p0 = _one_layer(3)
    g = _one_layer(4)
    lr, eps, T = 1e-3, 1e-8, 7
    p, state = p0, {}
    for t in range(1, T + 1):
        p = U.adamw(p, g, state, lr, t, eps=eps, wd=0.0)
    (w0, b0), (gw, gb), (wT, bT) = p0["l"], g["l"], p["l"]
    assert np.abs(wT - (w0 - T * lr * gw / (np.abs(gw) + eps))).max() < 1e-12
    assert np.abs(bT - (b0 - T * lr * gb / (np.abs(gb) + eps))).max() < 1e-12
    zero = {"l": (np.zeros_like(w0), np.zeros_like(b0))}
    p, state, wd = p0, {}, 0.05
    for t in range(1, T + 1):
        p = U.adamw(p, zero, state, lr, t, eps=eps, wd=wd)
    assert np.abs(p["l"][0] - w0 * (1 - lr * wd) ** T).max() < 1e-14
    assert np.array_equal(p["l"][1], b0)


def test_pool_and_upsample_by_hand():
    """2x2x2 mean pooling and nearest-neighbour 2x upsampling, entry by entry."""
    x = np.arange(4 * 4 * 4 * 2, dtype=float).reshape(4, 4, 4, 2)
    p = U.pool2(x)
    assert p.shape == (2, 2, 2, 2)
    for i in range(2):
        for j in range(2):
            for k in range(2):
                for c in range(2):
                    assert p[i, j, k, c] == x[2 * i:2 * i + 2, 2 * j:2 * j + 2, 2 * k:2 * k + 2, c].mean()
    u = U.up2(p)
    assert u.shape == x.shape
    for i in range(4):
        for j in range(4):
            for k in range(4):
                assert np.array_equal(u[i, j, k], p[i // 2, j // 2, k // 2])


def test_loss_is_the_mean_squared_error_of_the_corrected_start():
    """With a zero head the output is the start channel, so the loss is mean((x_start - target)^2)
    over every voxel; a head bias c adds c to every output."""
    params = U.init_params(7, c1=4)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((8, 8, 8, 5))
    t = rng.standard_normal((8, 8, 8, 1))
    assert U.loss(params, x, t) == pytest.approx(((x[..., -1:] - t) ** 2).mean(), rel=1e-14)
    w, _ = params["head"]
    params["head"] = (w, np.array([0.25]))
    assert U.loss(params, x, t) == pytest.approx(((x[..., -1:] + 0.25 - t) ** 2).mean(), rel=1e-14)
