"""The paper's own front end (Sec. 3, 3.2) on the GPU against the FP64 oracle: nearest-grid-point
binning, the radial number density n(r) of a survey, FKP weights 1/(1 + n P0) with P0 = 20000, a
random catalogue 100 times the galaxies, and the Eq. approx1 start."""
import numpy as np
import pytest

from oracle import recon_oracle as O
from paper_1504_02591_gb300 import mocks
from parity_helpers import mask_flips, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5
SHIFT_TOL = 1e-4


def test_ngp_deposit_vs_oracle(lib):
    from paper_1504_02591_gb300 import binding as B
    m = mocks.small_periodic(n_gal=200_000, n_ran=0, n_mesh=64)
    p = m.params()
    rng = np.random.default_rng(8)
    w = rng.uniform(0.5, 2.0, len(m.galaxies.pos)).astype(np.float32)
    r = B.Recon.from_mock(m, uniform=True)
    r.set_option(B.OPT_ASSIGN, B.ASSIGN_NGP)
    r.deposit(torch.from_numpy(m.galaxies.pos).cuda(), torch.from_numpy(w).cuda(), None, None)
    rho = r.get_field(B.FIELD_RHO_G).cpu().numpy()
    sw = r.scalars()["sum_wg"]
    r.close()
    ref = O.ngp_deposit(m.galaxies.pos, w.astype(np.float64), p["n"], p["L"])
    assert np.array_equal(rho != 0, ref != 0)          # the same node for every particle
    assert rel_l2(rho, ref) < 1e-6
    assert sw == pytest.approx(float(w.astype(np.float64).sum()), rel=1e-12)


@pytest.fixture(scope="module")
def survey100():
    """The survey shell at the 512^3 cell size on a 128^3 mesh, 100 randoms per galaxy (Sec. 3.2)."""
    return mocks.scaled_shell(128, 6.84 * 128, 15_000, 100, 1.87, 0.74, 77)


def test_radial_nbar_and_fkp_weights_vs_oracle(lib, survey100):
    from paper_1504_02591_gb300 import binding as B
    m = survey100
    p = m.params()
    w_ = m.window
    sky = 4 * np.pi * w_["sky_frac"]
    rmin, rmax, nb = w_["r_min"], w_["r_max"], 16
    r = B.Recon.from_mock(m)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    nbar = r.radial_nbar(gal, nb, rmin, rmax, sky)
    edges = np.linspace(rmin, rmax, nb + 1)
    want = O.radial_nbar(m.galaxies.pos, p["observer"], edges, sky)
    assert np.allclose(nbar, want, rtol=1e-12, atol=0)
    wg = r.fkp_weights(gal, nbar, rmin, rmax, 20000.0).cpu().numpy()
    wr = r.fkp_weights(ran, nbar, rmin, rmax, 20000.0).cpu().numpy()
    r.close()
    assert np.abs(wg - O.fkp_weights(m.galaxies.pos, p["observer"], edges, want)).max() < 1e-6
    assert np.abs(wr - O.fkp_weights(m.randoms.pos, p["observer"], edges, want)).max() < 1e-6


@pytest.mark.parametrize("ngp", [False, True])
def test_fkp_weighted_survey_vs_oracle(lib, survey100, ngp):
    """The whole reconstruction of an FKP-weighted survey with 100x randoms, binned with CIC or the
    paper's NGP, from the Eq. approx1 start, 4 updates, against the oracle given the same weights."""
    from paper_1504_02591_gb300 import binding as B
    m = survey100
    p = dict(m.params(), ngp=ngp)
    w_ = m.window
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    r = B.Recon.from_mock(m)
    nbar = r.radial_nbar(gal, 16, w_["r_min"], w_["r_max"], 4 * np.pi * w_["sky_frac"])
    wg = r.fkp_weights(gal, nbar, w_["r_min"], w_["r_max"])
    wr = r.fkp_weights(ran, nbar, w_["r_min"], w_["r_max"])
    if ngp:
        r.set_option(B.OPT_ASSIGN, B.ASSIGN_NGP)
    r.deposit(gal, wg, ran, wr)
    r.smooth()
    delta = r.get_field(B.FIELD_DELTA).cpu().numpy()
    r.iterate(B.START_APPROX1, 0.0, 4)
    psi = r.get_psi().cpu().numpy()
    sg = r.shift(gal, True).cpu().numpy()
    r.close()
    wg64 = wg.cpu().numpy().astype(np.float64)
    wr64 = wr.cpu().numpy().astype(np.float64)
    kw = dict(start=O.START_APPROX1, tol=0.0, max_iter=4)
    ref = O.reconstruct(p, m.galaxies.pos, wg64, m.randoms.pos, wr64, **kw)
    flips = mask_flips(ref, delta)          # decisions at the mask threshold, taken the GPU's way
    if len(flips):
        ref = O.reconstruct(p, m.galaxies.pos, wg64, m.randoms.pos, wr64, mask_flip=flips, **kw)
    e_d, e_p = rel_l2(delta, ref["delta"]), rel_l2(psi, ref["psi"])
    e_s = float(np.abs(sg - ref["shift_g"]).max())
    print(f"FKP survey (ngp={ngp}): delta {e_d:.2e}, Psi {e_p:.2e}, shift {e_s:.2e} Mpc/h")
    assert e_d < 1e-5 and e_p <= PSI_TOL and e_s <= SHIFT_TOL
