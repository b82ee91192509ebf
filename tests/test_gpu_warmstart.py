"""Learned warm start: the start plumbing (mesh and coarse levels) and what a trained network gains
over the analytic start."""
import numpy as np
import pytest

from oracle import recon_oracle as O
from oracle import unet_oracle as U
from paper_1504_02591_gb300 import mocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, L = 64, 437.5          # cell 6.84 Mpc/h, the 512^3 survey's resolution


def shell(seed, n_gal=2_500):
    return mocks.scaled_shell(N, L, n_gal, 50, 1.85, 0.74, seed)


def _prepared(B, m):
    r = B.Recon.from_mock(m)
    r.deposit(m.galaxies.pos, None, m.randoms.pos, None)
    r.smooth()
    return r


def _pool(a, f):
    n = a.shape[0]
    return a.reshape(n // f, f, n // f, f, n // f, f, *a.shape[3:]).mean(axis=(1, 3, 5))


def test_iterate_from_reproduces_analytic_start(lib):
    """Starting from the exported u_s of the Eq. approx2 start gives the Eq. approx2 iteration."""
    from paper_1504_02591_gb300 import binding as B
    r = _prepared(B, shell(300))
    feat = r.start_features(B.START_FFTA)
    u0 = feat[..., 4].contiguous()
    n1, rel1, _ = r.iterate_from(u0, 1e-6, 60)
    psi1, tr1 = r.get_psi().cpu().numpy(), np.array(r.trace())
    n2, rel2, _ = r.iterate(B.START_FFTA, 1e-6, 60)
    psi2, tr2 = r.get_psi().cpu().numpy(), np.array(r.trace())
    # the same start up to one float32 rounding of u_s: traces agree until the norms' noise floor
    assert abs(n1 - n2) <= 1
    big = tr2[: min(len(tr1), len(tr2))] > 1e-4
    assert np.allclose(tr1[: len(big)][big], tr2[: len(big)][big], rtol=1e-3)
    assert np.sqrt(((psi1 - psi2) ** 2).sum() / (psi2 ** 2).sum()) < 2e-6
    # starting from the converged radial displacement stops after (nearly) the minimum two updates
    u_conv = r.get_radial()
    n3, rel3, st3 = r.iterate_from(u_conv, 1e-6, 60)
    assert n3 <= 3 and rel3 < 1e-6 and st3 == B.OK
    psi3 = r.get_psi().cpu().numpy()
    assert np.sqrt(((psi3 - psi2) ** 2).sum() / (psi2 ** 2).sum()) < 2e-6
    r.close()


@pytest.mark.parametrize("level", [1, 2])
def test_coarse_start_with_zero_correction_is_the_analytic_start(lib, level):
    """u0 = the features' u_s channel adds exactly nothing: the iteration is bit for bit the
    Eq. approx2 iteration."""
    from paper_1504_02591_gb300 import binding as B
    r = _prepared(B, shell(301))
    feat = r.start_features(B.START_FFTA, level)
    assert feat.shape == (N >> level,) * 3 + (5,)
    n1, rel1, st1 = r.iterate_from(feat[..., 4].contiguous(), 1e-6, 60, level)
    psi1, tr1 = r.get_psi().cpu().numpy(), r.trace()
    n2, rel2, st2 = r.iterate(B.START_FFTA, 1e-6, 60)
    psi2, tr2 = r.get_psi().cpu().numpy(), r.trace()
    assert st1 == st2 == B.OK and n1 == n2
    assert tr1 == tr2
    assert np.array_equal(psi1, psi2)
    # the preparation is consumed
    with pytest.raises(B.ReconError):
        r.iterate_from(feat[..., 4].contiguous(), 1e-6, 60, level)
    r.close()


@pytest.mark.parametrize("level", [0, 1, 2])
def test_features_and_targets_match_oracle(lib, level):
    """Block means of delta, r and u_s = (1 - c) Psi_s . r, and of the converged Psi . r, against
    the FP64 oracle on a periodic box (no survey mask, so no threshold ambiguity)."""
    from paper_1504_02591_gb300 import binding as B
    m = mocks.small_periodic(n_gal=60_000, n_ran=0, n_mesh=64)
    p = m.params(uniform=True)
    ref = O.reconstruct(p, m.galaxies.pos, None, None, None, start=O.START_FFTA, tol=0.0, max_iter=8, shift=False)
    r = B.Recon.from_mock(m, uniform=True)
    r.deposit(m.galaxies.pos, None, None, None)
    r.smooth()
    feat = r.start_features(B.START_FFTA, level).cpu().numpy()
    r.iterate(B.START_FFTA, 0.0, 8)
    u_conv = r.get_radial(level).cpu().numpy()
    r.close()
    f = 1 << level
    rhat = np.moveaxis(O.rhat_field(p["n"], p["L"], p["observer"], p["los_mode"]), 0, -1)
    c = O.start_coefficient(O.START_FFTA, p["f"] / p["b"])
    psi_s = np.moveaxis(O.zeldovich(ref["delta"] / p["b"], p["L"]), 0, -1)
    want = np.concatenate([ref["delta"][..., None], rhat, (1 - c) * (psi_s * rhat).sum(-1, keepdims=True)], -1)
    want = _pool(want, f)
    for ch in range(5):
        err = np.sqrt(((feat[..., ch] - want[..., ch]) ** 2).sum() / (want[..., ch] ** 2).sum())
        assert err < 2e-5, (ch, err)
    u_ref = _pool((np.moveaxis(ref["psi"], 0, -1) * rhat).sum(-1), f)
    assert np.sqrt(((u_conv - u_ref) ** 2).sum() / (u_ref ** 2).sum()) < 1e-5


def test_trained_network_gains_over_analytic_start(lib):
    """Train the U-Net (the library's own forward/backward/AdamW kernels) on pairs the plain method
    produces at half resolution, then start held-out mocks from its prediction."""
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import warmstart as W
    level = 1
    pairs = [W.training_pair(shell(1000 + i), level) for i in range(8)]
    net = B.UNet(c1=8, bf16=True)
    net.set_params(B.flat_params(U.init_params(1, c1=8), U.layer_specs(8)))
    losses = W.train(net, pairs, steps=600, lr=2e-3)
    assert np.mean(losses[-30:]) < 0.9 * np.mean(losses[:8])
    gains = []
    for seed in (2000, 2001):
        m = shell(seed)
        feat, u_conv, n_ffta = W.training_pair(m, level)
        u_net = net.forward(feat)
        err_ffta = float(((feat[..., 4] - u_conv) ** 2).sum().sqrt() / (u_conv ** 2).sum().sqrt())
        err_net = float(((u_net - u_conv) ** 2).sum().sqrt() / (u_conv ** 2).sum().sqrt())
        r = _prepared(B, m)
        n_warm, rel, st = W.warm_iterate(r, net, level, 1e-6, 120)
        r.close()
        assert st == B.OK and rel < 1e-6
        gains.append((err_ffta, err_net, n_ffta, n_warm))
        print(f"held-out seed {seed}: coarse start error FFTA {err_ffta:.4f} learned {err_net:.4f}; "
              f"updates to 1e-6: FFTA {n_ffta} learned {n_warm}")
    # on held-out mocks the learned start is closer to the converged field than the analytic one,
    # and never needs more updates
    assert all(e_net < e_ffta for e_ffta, e_net, _, _ in gains), gains
    assert all(nw <= nf for _, _, nf, nw in gains), gains
    net.close()
