"""The warm-start U-Net kernels (forward, input and weight gradients, AdamW) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import unet_oracle as U

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(seed, n=8, c1=8):
    rng = np.random.default_rng(seed)
    params = U.init_params(seed, c1=c1)
    params["head"] = (rng.standard_normal((1, c1, 1)) * 0.3, np.array([0.05]))
    for k in params:
        w, b = params[k]
        params[k] = (w, b + 0.05 * rng.standard_normal(b.shape))
    x = rng.standard_normal((n, n, n, 5))
    target = rng.standard_normal((n, n, n, 1))
    return params, x, target


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


@pytest.mark.parametrize("n", [8, 16])
def test_unet_forward_and_gradients_fp32(lib, n):
    from paper_1504_02591_gb300 import binding as B
    c1 = 8
    params, x, target = _setup(11 + n, n=n, c1=c1)
    specs = U.layer_specs(c1)
    net = B.UNet(c1=c1, bf16=False)
    net.set_params(B.flat_params(params, specs))
    # the oracle sees the float32-rounded parameters and inputs the GPU sees
    p32 = B.unflat_params(B.flat_params(params, specs).astype(np.float64), specs)
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = target.astype(np.float32).astype(np.float64)
    y = net.forward(torch.from_numpy(x32.astype(np.float32))).cpu().numpy()
    y_ref, _ = U.forward(p32, x32)
    assert _rel(y, y_ref[..., 0]) < 1e-5
    loss = net.backward(torch.from_numpy(x32.astype(np.float32)), torch.from_numpy(t32[..., 0].astype(np.float32)))
    L_ref, g_ref = U.backward(p32, x32, t32)
    assert loss == pytest.approx(L_ref, rel=1e-5)
    g = B.unflat_params(net.get_grads().astype(np.float64), specs)
    for name, _, _ in specs:
        assert _rel(g[name][0], g_ref[name][0]) < 2e-4, name
        assert _rel(g[name][1], g_ref[name][1]) < 2e-4, name
    net.close()


def test_unet_forward_bf16(lib):
    from paper_1504_02591_gb300 import binding as B
    c1 = 16
    params, x, _ = _setup(5, n=16, c1=c1)
    specs = U.layer_specs(c1)
    net = B.UNet(c1=c1, bf16=True)
    net.set_params(B.flat_params(params, specs))
    y = net.forward(torch.from_numpy(x.astype(np.float32))).cpu().numpy()
    y_ref, _ = U.forward(params, x)
    # bfloat16 storage of weights and activations: ~3 significant digits
    assert _rel(y - x[..., -1], y_ref[..., 0] - x[..., -1]) < 3e-2
    net.close()


def test_unet_adamw_step_matches_oracle(lib):
    from paper_1504_02591_gb300 import binding as B
    c1 = 8
    params, x, target = _setup(21, n=8, c1=c1)
    specs = U.layer_specs(c1)
    net = B.UNet(c1=c1, bf16=False)
    net.set_params(B.flat_params(params, specs))
    p32 = B.unflat_params(B.flat_params(params, specs).astype(np.float64), specs)
    state = {}
    for step in (1, 2):
        net.backward(torch.from_numpy(x.astype(np.float32)), torch.from_numpy(target[..., 0].astype(np.float32)))
        g32 = B.unflat_params(net.get_grads().astype(np.float64), specs)
        net.adamw(1e-3, 1e-4)
        p32 = U.adamw(p32, g32, state, 1e-3, step, wd=1e-4)
    got = B.unflat_params(net.get_params().astype(np.float64), specs)
    for name, _, _ in specs:
        assert np.abs(got[name][0] - p32[name][0]).max() < 1e-6, name
    net.close()


def test_unet_training_reduces_loss(lib):
    from paper_1504_02591_gb300 import binding as B
    rng = np.random.default_rng(3)
    n = 16
    x = rng.standard_normal((n, n, n, 5)).astype(np.float32)
    # a smooth target the network can learn: a local linear function of the inputs
    target = (x[..., -1] + 0.5 * x[..., 0] - 0.2 * np.roll(x[..., 1], 1, axis=0)).astype(np.float32)
    net = B.UNet(c1=8, bf16=True)
    net.set_params(B.flat_params(U.init_params(7, c1=8), U.layer_specs(8)))
    xt, tt = torch.from_numpy(x), torch.from_numpy(target)
    first = net.backward(xt, tt)
    for _ in range(60):
        net.adamw(3e-3, 1e-4)
        last = net.backward(xt, tt)
    assert last < 0.5 * first
    net.close()
