"""Learned warm start: the start plumbing and what a trained network gains over the analytic start."""
import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_1504_02591_gb300 import mocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, L = 64, 437.5          # cell 6.84 Mpc/h, the 512^3 survey's resolution


def shell(seed, n_gal=2_500):
    return mocks.scaled_shell(N, L, n_gal, 50, 1.85, 0.74, seed)


def test_iterate_from_reproduces_analytic_start(lib):
    """Starting from the exported u_0 of the Eq. approx2 start gives the Eq. approx2 iteration."""
    from paper_1504_02591_gb300 import binding as B
    m = shell(300)
    r = B.Recon.from_mock(m)
    r.deposit(m.galaxies.pos, None, m.randoms.pos, None)
    r.smooth()
    feat = r.start_features(B.START_FFTA)
    u0 = feat[..., 4].contiguous()
    n1, rel1, _ = r.iterate_from(u0, 1e-6, 60)
    psi1, tr1 = r.get_psi().cpu().numpy(), np.array(r.trace())
    n2, rel2, _ = r.iterate(B.START_FFTA, 1e-6, 60)
    psi2, tr2 = r.get_psi().cpu().numpy(), np.array(r.trace())
    # the two starts differ only by the rounding of u_0 = (1 - c) Psi_s.r, so the traces agree
    # until they reach the float32 noise floor of the norms
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


def test_trained_network_gains_over_analytic_start(lib):
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import warmstart as W
    pairs = [W.training_pair(shell(1000 + i)) for i in range(6)]
    net = B.UNet(c1=8, bf16=True)
    net.set_params(B.flat_params(U.init_params(1, c1=8), U.layer_specs(8)))
    losses = W.train(net, pairs, steps=400, lr=2e-3)
    assert np.mean(losses[-30:]) < 0.9 * np.mean(losses[:6])
    gains = []
    for seed in (2000, 2001):
        m = shell(seed)
        feat, u_conv, n_ffta = W.training_pair(m)
        u_net = net.forward(feat)
        err_ffta = float(((feat[..., 4] - u_conv) ** 2).sum().sqrt() / (u_conv ** 2).sum().sqrt())
        err_net = float(((u_net - u_conv) ** 2).sum().sqrt() / (u_conv ** 2).sum().sqrt())
        r = B.Recon.from_mock(m)
        r.deposit(m.galaxies.pos, None, m.randoms.pos, None)
        r.smooth()
        n_warm, rel, st = W.warm_iterate(r, net, 1e-6, 120)
        r.close()
        assert st == B.OK and rel < 1e-6
        gains.append((err_ffta, err_net, n_ffta, n_warm))
        print(f"held-out seed {seed}: start error FFTA {err_ffta:.4f} learned {err_net:.4f}; "
              f"updates to 1e-6: FFTA {n_ffta} learned {n_warm}")
    # on held-out mocks the learned start is closer to the converged field than the analytic one,
    # and never needs more updates
    assert all(e_net < e_ffta for e_ffta, e_net, _, _ in gains), gains
    assert all(nw <= nf for _, _, nf, nw in gains), gains
    net.close()
