"""The benchmark workload at full size, run the way bench.py times it, against the FP64 oracle.

512^3 survey shell (6e5 galaxies, 3e7 randoms), learned warm start on the 4x coarsened mesh, the
iteration as one CUDA graph to 1e-6, then the shift of every galaxy and random.  The oracle cannot
iterate a 512^3 mesh in a test's time, so it checks what it can compute at this size:
  * the smoothed overdensity delta on every node (its own deposit, smoothing and survey mask);
  * that the converged Psi is a fixed point of Eq. iterative: one update computed by the oracle's
    operators in float64 from the GPU's delta and Psi returns Psi (the plain iteration's stopping
    rule and fixed point, whatever start the GPU took);
  * the shifts of sampled galaxies and randoms, gathered by the oracle from the GPU's Psi.
Tolerances are the ones the reconstruction is held to: rel L2 1e-5, shifts 1e-4 Mpc/h.
"""
import numpy as np
import pytest

from oracle import recon_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASK_BAND = 1e-5


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def test_benchmark_workload_full_size(lib):
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import mocks, warmstart
    m = mocks.survey_shell_512()
    p = m.params()
    n, L = p["n"], p["L"]
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    net, level = warmstart.load(warmstart.default_weights_path())
    r = B.Recon.from_mock(m)
    r.deposit(gal, None, ran, None)
    r.smooth()
    delta = r.get_field(B.FIELD_DELTA).cpu().numpy()
    feat = r.start_features(B.START_FFTA, level)
    n_it, rel, st = r.iterate_from(net.forward(feat), 1e-6, 80, level)
    assert st == B.OK and rel < 1e-6
    psi = r.get_psi().cpu().numpy()
    sg = r.shift(gal, True).cpu().numpy()
    sr = r.shift(ran, False).cpu().numpy()
    r.close()
    net.close()

    # delta: deposit, smoothing and mask of the oracle on the full mesh
    rho_r = O.cic_deposit(m.randoms.pos, None, n, L)
    n_touched = int(np.count_nonzero(rho_r > 0))
    rho_r_s = O.smooth(rho_r, p["R"], L)
    del rho_r
    rho_g_s = O.smooth(O.cic_deposit(m.galaxies.pos, None, n, L), p["R"], L)
    d_ref, mask, alpha, thr = O.overdensity_randoms(rho_g_s, rho_r_s, float(len(m.galaxies.pos)),
                                                    float(len(m.randoms.pos)), p["mask_frac"], n_touched)
    del rho_g_s
    gmask = delta != 0
    flips = gmask != mask
    # the mask is a floating-point decision: the GPU may take either branch only at the threshold
    assert np.all(np.abs(rho_r_s[flips] - thr) <= MASK_BAND * thr), int(flips.sum())
    del rho_r_s
    keep = ~flips
    e_delta = _rel(delta[keep], d_ref[keep])
    print(f"512^3: {int(flips.sum())} mask decisions at the threshold, delta rel L2 {e_delta:.2e}")
    assert e_delta < 1e-5
    del d_ref, mask, gmask, flips, keep

    # fixed point of Eq. iterative: Z[delta/b + beta div((Psi.r) r)] = Psi
    beta = p["f"] / p["b"]
    rhat = O.rhat_field(n, L, p["observer"], p["los_mode"])
    S_k = O.fft3(delta.astype(np.float64) / p["b"]) + beta * O.divergence(
        O.radial_projection(psi.astype(np.float64), rhat), L)
    psi_next = np.stack([O.ifft3(c_k, n) for c_k in O.zeldovich_k(S_k, n, L)])
    del S_k, rhat
    e_fix = _rel(psi, psi_next)
    print(f"512^3: {n_it} updates, last rel {rel:.2e}, fixed-point rel L2 {e_fix:.2e}")
    assert e_fix < 1e-5

    # shifts of sampled tracers, gathered by the oracle from the GPU's Psi
    rng = np.random.default_rng(0)
    ig = rng.choice(len(m.galaxies.pos), 20_000, replace=False)
    ir = rng.choice(len(m.randoms.pos), 20_000, replace=False)
    psi64 = psi.astype(np.float64)
    dg = O.shift_vectors(psi64, m.galaxies.pos[ig], L, p["f"], p["observer"], p["los_mode"], True)
    dr = O.shift_vectors(psi64, m.randoms.pos[ir], L, p["f"], p["observer"], p["los_mode"], False)
    e_g, e_r = float(np.abs(sg[ig] - dg).max()), float(np.abs(sr[ir] - dr).max())
    print(f"512^3: max shift error galaxies {e_g:.2e}, randoms {e_r:.2e} Mpc/h")
    assert e_g <= 1e-4 and e_r <= 1e-4
