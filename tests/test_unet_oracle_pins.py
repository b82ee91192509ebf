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
