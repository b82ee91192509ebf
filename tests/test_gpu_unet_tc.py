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


def _bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return r.view(np.float32)


def _bf16_ulp(v):
    """Spacing of bfloat16 numbers (8 significant bits) at |v|."""
    a = np.maximum(np.abs(v), 1e-30)
    return np.exp2(np.floor(np.log2(a)) - 7)


@pytest.mark.parametrize("n,c1", [(128, 8), (128, 16)])
def test_tensor_core_forward_layers_vs_fp64_oracle(lib, n, c1):
    """Each layer of the tensor-core forward against the FP64 oracle's convolution (Eq.-free: the
    network has no counterpart in the paper) given the same inputs: the GPU's own stored bf16 input
    activations (so errors do not compound), the weights rounded to bf16 as the GPU stores them and
    the float32 biases.  Every output must be the bf16 rounding of the exact value up to one bf16
    unit (float32 sums may round the other way at a tie) plus float32 summation error; a wrong
    operand layout, tap offset or channel group gives O(1) errors.  The fused 1x1 head and residual
    of the last layer are checked on the float32 network output."""
    from paper_1504_02591_gb300 import binding as B
    specs = U.layer_specs(c1)
    rng = np.random.default_rng(90 + c1)
    params = U.init_params(90 + c1, c1=c1)
    params["head"] = (rng.standard_normal((1, c1, 1)) * 0.3, np.array([0.05]))
    for k in params:
        w, b = params[k]
        params[k] = (w, b + 0.05 * rng.standard_normal(b.shape))
    flat = B.flat_params(params, specs)
    gp = B.unflat_params(flat, specs)                  # float32 values the GPU holds
    wq = {k: (_bf16(w).astype(np.float64), b.astype(np.float64)) for k, (w, b) in gp.items()}
    net = B.UNet(c1=c1, bf16=True)
    net.set_params(flat)
    g = torch.Generator().manual_seed(7 * n + c1)
    x = torch.randn((n, n, n, 5), generator=g)
    y = net.forward(x.cuda()).cpu().numpy().astype(np.float64)
    side = [n, n, n // 2, n // 2, n // 4, n // 4, n // 2, n // 2, n, n]
    act = {l: net.get_layer(l, side[l], specs[l][2]).astype(np.float64) for l in range(9)}
    net.close()
    x64 = x.numpy().astype(np.float64)
    pool = lambda a: _bf16(U.pool2(a)).astype(np.float64)      # the GPU stores pooled maps in bf16
    inputs = {
        0: _bf16(x.numpy()).astype(np.float64), 1: act[0], 2: pool(act[1]), 3: act[2], 4: pool(act[3]),
        5: act[4], 6: np.concatenate([U.up2(act[5]), act[3]], axis=3), 7: act[6],
        8: np.concatenate([U.up2(act[7]), act[1]], axis=3),
    }
    for l in range(9):
        name = specs[l][0]
        exact = np.maximum(U.conv3(inputs[l], *wq[name]), 0.0)
        err = np.abs(act[l] - exact)
        bound = _bf16_ulp(exact) + 1e-4 * np.abs(exact).max()
        off = int((err > bound).sum())
        flips = float((act[l] != _bf16(exact)).mean())
        print(f"n={n} c1={c1} {name}: max err/bound {float((err / bound).max()):.2f}, "
              f"{100 * flips:.3f}% elements one unit off the exact rounding")
        assert off == 0, (name, off)
        assert flips < 0.01, (name, flips)
    d1b = _bf16(np.maximum(U.conv3(act[8], *wq["dec1b"]), 0.0)).astype(np.float64)
    hw, hb = wq["head"]
    want = U.conv3(d1b, hw, hb)[..., 0] + x64[..., 4]
    e = _rel(y - x64[..., 4], want - x64[..., 4])
    print(f"n={n} c1={c1} fused head + residual: rel L2 {e:.2e}")
    assert e < 2e-3
