"""Tensor-core (tcgen05) U-Net forward against the CUDA-core forward, layer by layer.

Both paths store every activation as bfloat16 at the same points and sum in float32, so they differ
only where a float32 sum taken in another order rounds to a neighbouring bfloat16: a handful of
elements by one bf16 unit.  A wrong operand layout, tap offset or channel group gives O(1) errors.
The CUDA-core path itself is checked against the FP64 oracle in test_gpu_unet.py.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-30)))


def _net(B, c1, seed):
    rng = np.random.default_rng(seed)
    params = U.init_params(seed, c1=c1)
    params["head"] = (rng.standard_normal((1, c1, 1)) * 0.3, np.array([0.05]))
    for k in params:
        w, b = params[k]
        params[k] = (w, b + 0.05 * rng.standard_normal(b.shape))
    net = B.UNet(c1=c1, bf16=True)
    net.set_params(B.flat_params(params, U.layer_specs(c1)))
    return net


# n = 128: level 1 on z runs of 128 (M = voxels), level 2 on runs of 64 (M = output channels),
# level 3 (32^3) on the CUDA cores.  n = 256 adds a second z block per row and level 3 at 64.
@pytest.mark.parametrize("n,c1", [(128, 8), (128, 16), (256, 8)])
def test_tensor_core_forward_matches_cuda_core(lib, n, c1):
    from paper_1504_02591_gb300 import binding as B
    net = _net(B, c1, 40 + c1)
    g = torch.Generator().manual_seed(n + c1)
    x = torch.randn((n, n, n, 5), generator=g).cuda()
    specs = U.layer_specs(c1)
    level = [0, 0, 1, 1, 2, 2, 1, 1, 0, 0]
    net.set_option(B.UNET_OPT_TENSOR_CORES, 0)
    y_ref = net.forward(x).cpu().numpy()
    ref = [net.get_layer(l, n >> level[l], specs[l][2]) for l in range(10)]
    net.set_option(B.UNET_OPT_TENSOR_CORES, 1)
    y_tc = net.forward(x).cpu().numpy()
    x4 = x[..., 4].cpu().numpy()
    errs = [_rel(net.get_layer(l, n >> level[l], specs[l][2]), ref[l]) for l in range(9)]
    print(f"n={n} c1={c1} per-layer rel L2:", " ".join(f"{e:.1e}" for e in errs))
    # one-unit bf16 flips enter at every layer and compound with depth (measured ~3e-4 per layer)
    for l, e in enumerate(errs):
        assert e < 1e-3 * (l + 1), (l, specs[l][0], e)
    assert _rel(y_tc - x4, y_ref - x4) < 1e-2
    # a second call reuses the packed weights and must agree exactly with the first
    y_tc2 = net.forward(x).cpu().numpy()
    assert np.array_equal(y_tc, y_tc2)
    net.close()


def test_tensor_core_forward_after_training_step(lib):
    """The packed weight tiles follow AdamW updates."""
    from paper_1504_02591_gb300 import binding as B
    n, c1 = 128, 8
    net = _net(B, c1, 7)
    g = torch.Generator().manual_seed(3)
    x = torch.randn((n, n, n, 5), generator=g).cuda()
    t = torch.randn((n, n, n), generator=g).cuda()
    net.forward(x)
    net.backward(x, t)
    net.adamw(1e-2, 1e-4)
    y_tc = net.forward(x).cpu().numpy()
    net.set_option(B.UNET_OPT_TENSOR_CORES, 0)
    y_ref = net.forward(x).cpu().numpy()
    x4 = x[..., 4].cpu().numpy()
    assert _rel(y_tc - x4, y_ref - x4) < 1e-2
    net.close()
