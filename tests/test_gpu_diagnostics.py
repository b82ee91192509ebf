"""The paper's diagnostics on the GPU against the FP64 oracle.

* The plane-parallel Helmholtz split of Sec. 4.1 (Eq. Helmholtz, Eq. irrotational, Eq. solenoidal)
  of a reconstructed displacement, and the statistics of the ratio of its x components.
* The radial ratio of Eq. ratio (Sec. 4.3, 5.2; Tables 1-3): the displacement of the real-space
  galaxies over an estimate from the redshift-space galaxies, both projected on each galaxy's line of
  sight, with the paper's outlier rule (ratios above 3 or below -1 cut).
* The convergence pattern of Sec. 5.2 on a synthetic Zel'dovich survey: from the uncorrected start
  the mean ratio oscillates about 1 and settles later than from the Eq. approx2 start.
"""
import numpy as np
import pytest

from oracle import recon_oracle as O
from paper_1504_02591_gb300 import mocks
from parity_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shell():
    return mocks.survey_shell_512(n_gal=60_000, ran_ratio=50, n_mesh=128)


def _psi(B, m, pos, f, start, n_it):
    """GPU displacement after n_it updates for the galaxies at pos (the mock's randoms and options)."""
    r = B.Recon.from_mock(m, f=f)
    r.deposit(torch.from_numpy(pos).cuda(), None, torch.from_numpy(m.randoms.pos).cuda(), None)
    r.smooth()
    r.iterate(start, 0.0, n_it)
    psi = r.get_psi()
    r.close()
    return psi


def test_helmholtz_split_vs_oracle(lib, shell):
    from paper_1504_02591_gb300 import binding as B
    m = shell
    p = m.params()
    psi = _psi(B, m, m.galaxies.pos, p["f"], B.START_FFTA, 3)
    r = B.Recon.from_mock(m)
    ga, cb = r.helmholtz_x(psi[0])
    want_ga, want_cb = O.helmholtz_x(psi.cpu().numpy().astype(np.float64), p["L"])
    e_ga, e_cb = rel_l2(ga.cpu().numpy(), want_ga), rel_l2(cb.cpu().numpy(), want_cb)
    # statistics of the irrotational / solenoidal ratio per axis, without and with the outlier cut
    for j in range(3):
        for lo, hi in ((-1e300, 1e300), (O.RATIO_LO, O.RATIO_HI)):
            got = r.ratio_stats(ga[j], cb[j], lo, hi)
            want = O.ratio_stats(ga[j].cpu().numpy(), cb[j].cpu().numpy(), lo, hi)
            assert got[3] == want[3] and got[2] == pytest.approx(want[2], abs=1e-12)
            assert got[0] == pytest.approx(want[0], rel=1e-9, abs=1e-9)
            assert got[1] == pytest.approx(want[1], rel=1e-6)
    x = r.ratio_stats(ga[0], cb[0])
    r.close()
    print(f"Helmholtz split 128^3: grad A rel L2 {e_ga:.2e}, curl B {e_cb:.2e}; x ratio mean {x[0]:.3f} "
          f"sigma {x[1]:.3f} ({100 * x[2]:.1f}% cut)")
    assert e_ga < 1e-5 and e_cb < 1e-5


def test_radial_ratio_vs_oracle(lib):
    from paper_1504_02591_gb300 import binding as B
    m = mocks.small_periodic(n_gal=100_000, n_ran=1_000_000, n_mesh=64)
    p = m.params()
    real = _psi(B, m, m.galaxies_real.pos, 0.0, B.START_PLAIN, 1)     # Psi_real,FFT = Z[delta_real/b]
    est = _psi(B, m, m.galaxies.pos, p["f"], B.START_FFTA, 2)
    r = B.Recon.from_mock(m)
    got = r.radial_ratio(real, est, torch.from_numpy(m.galaxies.pos).cuda())
    r.close()
    ref_real = O.reconstruct(dict(p, f=0.0), m.galaxies_real.pos, None, m.randoms.pos, None, start=O.START_PLAIN,
                             tol=0.0, max_iter=1, shift=False)
    ref_est = O.reconstruct(p, m.galaxies.pos, None, m.randoms.pos, None, start=O.START_FFTA, tol=0.0,
                            max_iter=2, shift=False)
    want = O.radial_ratio(ref_real["psi"], ref_est["psi"], m.galaxies.pos, p["L"], p["observer"], p["los_mode"],
                          periodic=True)
    print(f"radial ratio 64^3: GPU {got}, oracle {want}")
    assert got[0] == pytest.approx(want[0], rel=1e-4)
    assert got[1] == pytest.approx(want[1], rel=1e-3)
    assert abs(got[3] - want[3]) <= 1e-3 * len(m.galaxies.pos)


def _iterate_ratios(B, m, start, n_max, real):
    """Mean radial ratio (Psi_real . r)/(Psi_n . r) at the galaxies for n = 0 .. n_max."""
    p = m.params()
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    out = []
    r = B.Recon.from_mock(m)
    r.deposit(gal, None, torch.from_numpy(m.randoms.pos).cuda(), None)
    r.smooth()
    # n = 0: the start itself; its radial component is (1 - c) Z[delta/b].r
    beta = p["f"] / p["b"]
    c = O.start_coefficient(start, beta)
    r0 = B.Recon.from_mock(m, f=0.0)       # with f = 0 one update returns Z[delta/b] of the same delta
    r0.deposit(gal, None, torch.from_numpy(m.randoms.pos).cuda(), None)
    r0.smooth()
    r0.iterate(B.START_PLAIN, 0.0, 1)
    psi_s = r0.get_psi()
    r0.close()
    out.append(r.radial_ratio(real, (1.0 - c) * psi_s, gal)[:3])
    for n in range(1, n_max + 1):
        r.iterate(start, 0.0, n)
        out.append(r.radial_ratio(real, r.get_psi(), gal)[:3])
    r.close()
    return out


def test_convergence_pattern_of_the_radial_ratio(lib):
    """Sec. 5.2 (Tables 2-3) on a 128^3 survey shell whose spectrum turns over at k = 0.02 h/Mpc:
    from the uncorrected start the mean ratio starts below its converged value (the redshift-space
    displacement is too large) and oscillates about it; the Eq. approx2 start begins closer and
    converges (the rule of Sec. 5.2) no later; the limit is 1 within 2%, as in the paper's tables.
    (With the benchmark's k^-1.5 spectrum the limit sits near 0.77: bulk flows from scales larger
    than the window move the galaxies in redshift space, and no solve inside the window sees them.)"""
    from paper_1504_02591_gb300 import binding as B
    m = mocks.survey_shell_512(n_gal=60_000, ran_ratio=50, n_mesh=128, amp=1.0, seed=40, k_turn=0.02)
    real = _psi(B, m, m.galaxies_real.pos, 0.0, B.START_PLAIN, 1)
    plain = _iterate_ratios(B, m, B.START_PLAIN, 7, real)
    ffta = _iterate_ratios(B, m, B.START_FFTA, 7, real)
    mp, mf = [x[0] for x in plain], [x[0] for x in ffta]
    print("n  plain(mean, sigma, cut)  FFTA(mean, sigma, cut)")
    for n in range(len(mp)):
        print(n, np.round(plain[n], 3), np.round(ffta[n], 3))
    cp, cf = O.converged_at(mp), O.converged_at(mf)
    print(f"converged (Sec. 5.2 rule): uncorrected start n = {cp}, Eq. approx2 start n = {cf}")
    lim = mp[-1]
    assert abs(lim - 1.0) < 0.02
    assert abs(mf[-1] - lim) < 1e-3 * abs(lim)          # both starts reach the same fixed point
    assert mp[0] < lim and abs(mf[0] - lim) < abs(mp[0] - lim)
    assert (mp[0] - lim) * (mp[1] - lim) < 0 and (mp[1] - lim) * (mp[2] - lim) < 0   # oscillation
    assert cf <= cp
