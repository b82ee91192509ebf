"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded synthetic inputs.

Tolerances (stated by the method's precision policy): relative L2 error of Psi <= 1e-5 and maximum
particle-shift error <= 1e-4 Mpc/h against the FP64 oracle.  Intermediate fields are checked at the
float32 rounding level they are computed at.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import recon_oracle as O
from paper_1504_02591_gb300 import mocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5
SHIFT_TOL = 1e-4


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_02591_gb300 import binding
    return binding


# ------------------------------------------------------------------------------------------------
# Spectral engine alone
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [32, 48, 64, 96, 128])
def test_fft_r2c_c2r_vs_oracle(B, n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, n, n))
    r = B.Recon(n, 1000.0, 2.0, 0.7, 10.0, (0, 0, 0), uniform=True)
    X = r.fft_r2c(torch.from_numpy(x.astype(np.float32))).cpu().numpy().astype(np.complex128)
    want = O.fft3(x.astype(np.float32).astype(np.float64))
    assert np.abs(X - want).max() <= 2e-6 * np.abs(want).max()
    assert rel_l2(X.view(np.float64), want.view(np.float64)) <= 1e-6
    # c2r of the exact spectrum is N^3 times the inverse transform
    y = r.fft_c2r(torch.from_numpy(want.astype(np.complex64))).cpu().numpy()
    assert rel_l2(y / n ** 3, x.astype(np.float32)) <= 1e-6
    r.close()


# ------------------------------------------------------------------------------------------------
# Whole pipeline, small periodic box (64^3, 2e5 galaxies, 2e6 randoms, radial LOS)
# ------------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def periodic_mock():
    return mocks.small_periodic()


@pytest.fixture(scope="module")
def periodic_oracle(periodic_mock):
    m = periodic_mock
    out = {}
    for start in (O.START_PLAIN, O.START_APPROX1, O.START_FFTA):
        out[start] = O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos, None,
                                   start=start, tol=0.0, max_iter=6)
    return out


@pytest.mark.parametrize("start", [0, 1, 2])
def test_periodic_pipeline_vs_oracle(B, periodic_mock, periodic_oracle, start):
    m = periodic_mock
    ref = periodic_oracle[start]
    r = B.Recon.from_mock(m)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    r.deposit(gal, None, ran, None)
    rho_g = r.get_field(B.FIELD_RHO_G).cpu().numpy()
    assert rel_l2(rho_g, ref["rho_g"]) < 1e-6
    assert abs(rho_g.astype(np.float64).sum() - len(m.galaxies.pos)) < 1e-5 * len(m.galaxies.pos)
    r.smooth()
    sc = r.scalars()
    assert sc["sum_wg"] == len(m.galaxies.pos) and sc["sum_wr"] == len(m.randoms.pos)
    assert sc["threshold"] == pytest.approx(ref["threshold"], rel=1e-12)
    delta = r.get_field(B.FIELD_DELTA).cpu().numpy()
    assert rel_l2(delta, ref["delta"]) < 2e-6
    n_it, rel, st = r.iterate(start, 0.0, 6)
    assert n_it == 6 and st == B.OK
    tr = np.array(r.trace())
    assert np.allclose(tr, ref["rel"], rtol=1e-3, atol=0)
    psi = r.get_psi().cpu().numpy()
    assert rel_l2(psi, ref["psi"]) <= PSI_TOL
    sg = r.shift(gal, True).cpu().numpy()
    sr = r.shift(ran, False).cpu().numpy()
    assert np.abs(sg - ref["shift_g"]).max() <= SHIFT_TOL
    assert np.abs(sr - ref["shift_r"]).max() <= SHIFT_TOL
    # host-memory catalogue and outputs give the same shifts and wrapped positions
    sh_h, po_h = r.shift(m.galaxies.pos, True, want_pos=True)
    assert np.array_equal(sh_h, sg)
    assert np.abs(po_h - ref["pos_g"]).max() <= SHIFT_TOL
    r.close()


@pytest.mark.parametrize("dep_path,shift_path", [(0, 1), (1, 0), (1, 1)])
def test_particle_paths_vs_oracle(B, periodic_mock, periodic_oracle, dep_path, shift_path):
    """Direct and brick-sorted deposit / shift paths give the oracle's densities and shifts."""
    m = periodic_mock
    ref = periodic_oracle[2]
    r = B.Recon.from_mock(m)
    r.set_option(B.OPT_DEPOSIT_PATH, dep_path)
    r.set_option(B.OPT_SHIFT_PATH, shift_path)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    r.deposit(gal, None, ran, None)
    assert rel_l2(r.get_field(B.FIELD_RHO_G).cpu().numpy(), ref["rho_g"]) < 1e-6
    assert rel_l2(r.get_field(B.FIELD_RHO_R).cpu().numpy(), ref["rho_r"]) < 1e-6
    r.smooth()
    r.iterate(2, 0.0, 6)
    assert rel_l2(r.get_psi().cpu().numpy(), ref["psi"]) <= PSI_TOL
    sg, pg = r.shift(gal, True, want_pos=True)
    sr = r.shift(ran, False)
    assert np.abs(sg.cpu().numpy() - ref["shift_g"]).max() <= SHIFT_TOL
    assert np.abs(sr.cpu().numpy() - ref["shift_r"]).max() <= SHIFT_TOL
    assert np.abs(pg.cpu().numpy() - ref["pos_g"]).max() <= SHIFT_TOL
    r.close()


def test_graph_and_host_loops_agree(B, shell_case):
    """The device-driven loop (one CUDA graph, conditional WHILE node) and the host-driven loop run
    the same kernels on the same delta(k): they stop at the same update with the same trace and Psi."""
    m, ref = shell_case
    r = B.Recon.from_mock(m)
    r.deposit(torch.from_numpy(m.galaxies.pos).cuda(), None, torch.from_numpy(m.randoms.pos).cuda(), None)
    r.smooth()
    out = {}
    for graph in (1, 0):
        r.set_option(B.OPT_GRAPH, graph)
        n_it, rel, st = r.iterate(2, 1e-6, 40)
        out[graph] = (n_it, np.array(r.trace()), r.get_psi().cpu().numpy(), st)
    r.close()
    assert out[1][0] == out[0][0] and out[1][3] == out[0][3] == B.OK
    assert np.array_equal(out[1][1], out[0][1])
    assert np.array_equal(out[1][2], out[0][2])
    # max_iter caps the device loop too
    r = B.Recon.from_mock(m)
    n_it, rel, st = r.run(m.galaxies.pos, m.randoms.pos, start=0, tol=1e-12, max_iter=3)
    assert n_it == 3 and st == B.ERR_NOT_CONVERGED and len(r.trace()) == 3
    r.close()


def test_delta_k_export_matches_oracle(B, periodic_mock, periodic_oracle):
    m = periodic_mock
    r = B.Recon.from_mock(m)
    r.run(m.galaxies.pos, m.randoms.pos, start=0, tol=0, max_iter=2)
    dk = r.get_field(B.FIELD_DELTA_K).cpu().numpy()
    want = O.fft3(periodic_oracle[0]["delta"])
    assert rel_l2(dk.view(np.float32).astype(np.float64), want.view(np.float64)) < 3e-6
    r.close()


# ------------------------------------------------------------------------------------------------
# Survey shell with mask (the 512^3 survey shape scaled to 128^3 and 6e4 galaxies)
# ------------------------------------------------------------------------------------------------
MASK_BAND = 1e-5   # relative distance to the mask threshold within which either decision is valid


def mask_ambiguity(ref):
    """Flat indices of nodes whose FP64 smoothed random density is within MASK_BAND of the threshold."""
    rr = ref["rho_r_s"].reshape(-1)
    return np.nonzero(np.abs(rr - ref["threshold"]) <= MASK_BAND * ref["threshold"])[0]


def check_mask_and_rerun(m, ref, gpu_delta, start, tol, max_iter):
    """The GPU mask (nodes where its delta is nonzero) may differ from the oracle's only at nodes
    within rounding of the threshold; if it does, the oracle is rerun with those decisions taken
    the GPU's way (each is a valid branch) so the comparison is against the same branch."""
    gmask = (gpu_delta != 0).reshape(-1)
    omask = ref["mask"].reshape(-1)
    diff = np.nonzero(gmask != omask)[0]
    amb = set(mask_ambiguity(ref).tolist())
    assert all(int(i) in amb for i in diff), f"{len(diff)} mask differences, not all at the threshold"
    if len(diff) == 0:
        return ref
    return O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos, None, start=start, tol=tol,
                         max_iter=max_iter, mask_flip=diff)


@pytest.fixture(scope="module")
def shell_case():
    m = mocks.survey_shell_512(n_gal=60_000, ran_ratio=50, n_mesh=128)
    ref = O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos, None,
                        start=O.START_FFTA, tol=1e-6, max_iter=40)
    return m, ref


def test_shell_survey_converged_vs_oracle(B, shell_case):
    m, ref = shell_case
    r = B.Recon.from_mock(m)
    r.deposit(torch.from_numpy(m.galaxies.pos).cuda(), None, torch.from_numpy(m.randoms.pos).cuda(), None)
    r.smooth()
    sc = r.scalars()
    assert sc["threshold"] == pytest.approx(ref["threshold"], rel=1e-12)
    delta = r.get_field(B.FIELD_DELTA).cpu().numpy()
    ref = check_mask_and_rerun(m, ref, delta, O.START_FFTA, 1e-6, 40)
    assert rel_l2(delta, ref["delta"]) < 1e-5
    n_it, rel, st = r.iterate(2, 1e-6, 40)
    assert st == B.OK and rel < 1e-6
    assert abs(n_it - ref["n_iter"]) <= 1
    psi = r.get_psi().cpu().numpy()
    assert rel_l2(psi, ref["psi"]) <= PSI_TOL
    sg = r.shift(torch.from_numpy(m.galaxies.pos).cuda(), True).cpu().numpy()
    assert np.abs(sg - ref["shift_g"]).max() <= SHIFT_TOL
    sr = r.shift(torch.from_numpy(m.randoms.pos).cuda(), False).cpu().numpy()
    assert np.abs(sr - ref["shift_r"]).max() <= SHIFT_TOL
    r.close()


@pytest.mark.parametrize("host", [False, True])
def test_retained_sort_shift(B, shell_case, host):
    """RECON_OPT_REUSE_SORT: the random shift reuses the sorted deposit's brick order (no second sort,
    no second read of the positions; page-locked host catalogues are sorted in place) and gives the
    shifts of the default path; the galaxy shift meanwhile takes the direct path."""
    m, ref = shell_case
    if host:
        gal = torch.from_numpy(m.galaxies.pos).pin_memory()
        ran = torch.from_numpy(m.randoms.pos).pin_memory()
    else:
        gal = torch.from_numpy(m.galaxies.pos).cuda()
        ran = torch.from_numpy(m.randoms.pos).cuda()
    out = {}
    for reuse in (0, 1):
        r = B.Recon.from_mock(m)
        # both runs deposit through the brick sort (the same fixed-point positions, so the same mask
        # decisions); the first sorts again for its shifts, the second reuses the deposit's order
        r.set_option(B.OPT_DEPOSIT_PATH, B.PATH_SORTED)
        if reuse:
            r.set_option(B.OPT_REUSE_SORT, 1)
        r.deposit(gal, None, ran, None)
        r.smooth()
        # a fixed number of updates: both runs stop at the same one (with a tolerance the stopping
        # update itself may differ, a 1e-6 relative change of Psi)
        n_it, rel, st = r.iterate(B.START_FFTA, 0.0, 12)
        assert st == B.OK and n_it == 12
        sg = r.shift(gal, True)
        sorts = r.timing()["sort"][0]
        sr = r.shift(ran, False)
        if reuse:
            assert r.timing()["sort"][0] == sorts      # the random shift sorted nothing
        out[reuse] = (np.asarray(sg.cpu() if hasattr(sg, "cpu") else sg),
                      np.asarray(sr.cpu() if hasattr(sr, "cpu") else sr))
        r.close()
    # the two deposits differ only in the order of their float32 sums; the galaxy shifts in path
    # (sorted, then direct)
    assert np.abs(out[1][0] - out[0][0]).max() <= SHIFT_TOL
    assert np.abs(out[1][1] - out[0][1]).max() <= SHIFT_TOL


# ------------------------------------------------------------------------------------------------
# Uniform mean density, fixed LOS and lognormal (the large periodic run's options, at 64^3)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("los_mode,lognormal", [(1, False), (0, True), (1, True)])
def test_uniform_options_vs_oracle(B, los_mode, lognormal):
    obs = (1.0, 0.0, 0.0) if los_mode == 1 else (-1000.0, 1250.0, 1250.0)
    m = mocks.periodic_box(2500.0, 64, 150_000, 0, 1.0, 0.74, 40.0, obs, 20, 21, 22, ng=64,
                           los_mode=los_mode, uniform=True)
    p = m.params(lognormal=lognormal)
    ref = O.reconstruct(p, m.galaxies.pos, None, None, None, start=O.START_FFTA, tol=0.0, max_iter=6)
    r = B.Recon.from_mock(m, lognormal=lognormal)
    r.run(torch.from_numpy(m.galaxies.pos).cuda(), None, start=2, tol=0.0, max_iter=6)
    psi = r.get_psi().cpu().numpy()
    assert rel_l2(psi, ref["psi"]) <= PSI_TOL
    sg = r.shift(torch.from_numpy(m.galaxies.pos).cuda(), True).cpu().numpy()
    assert np.abs(sg - ref["shift_g"]).max() <= SHIFT_TOL
    if lognormal:
        assert r.scalars()["lognormal_C"] == pytest.approx(ref["lognormal_C"], rel=1e-4)
    r.close()


# ------------------------------------------------------------------------------------------------
# Edge cases and errors
# ------------------------------------------------------------------------------------------------
def test_state_and_argument_errors(B):
    r = B.Recon(32, 500.0, 2.0, 0.7, 10.0, (600.0, 250.0, 250.0))
    with pytest.raises(B.ReconError) as e:
        r.smooth()
    assert e.value.status == B.ERR_STATE
    with pytest.raises(B.ReconError) as e:
        r.deposit(np.zeros((0, 3)), None, np.random.default_rng(0).uniform(0, 500, (100, 3)))
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.ReconError) as e:
        r.deposit(np.random.default_rng(0).uniform(0, 500, (100, 3)), None, None)
    assert e.value.status == B.ERR_INVALID_ARG
    r.close()


def test_not_converged_reports_status(B):
    m = mocks.small_periodic(n_gal=20_000, n_ran=200_000, n_mesh=32)
    r = B.Recon.from_mock(m)
    n_it, rel, st = r.run(m.galaxies.pos, m.randoms.pos, start=0, tol=1e-12, max_iter=3)
    assert n_it == 3 and st == B.ERR_NOT_CONVERGED and rel > 1e-12
    r.close()


def test_ragged_particle_counts(B):
    """Counts that are not multiples of the block size or the staging chunk."""
    rng = np.random.default_rng(5)
    gal = rng.uniform(0, 500.0, (1, 3))
    ran = rng.uniform(0, 500.0, (2_097_152 + 37, 3))
    r = B.Recon(32, 500.0, 2.0, 0.7, 20.0, (250.0, 250.0, 250.0), periodic=True)
    r.deposit(gal, None, ran, None)
    rho_r = r.get_field(B.FIELD_RHO_R).cpu().numpy()
    assert abs(rho_r.astype(np.float64).sum() - len(ran)) <= 1e-5 * len(ran)
    want = O.cic_deposit(ran, None, 32, 500.0)
    assert rel_l2(rho_r, want) < 1e-6
    r.close()


def test_particle_edge_positions(B):
    """Positions on nodes, just below a node (fractions that round up to a whole cell), at 0, -0 and
    L, negative and beyond the box (periodic images, whose line of sight runs to the image in
    [0, L)): both deposit and both shift paths against the oracle's CIC on the same positions."""
    n, L = 32, 500.0
    h = L / n
    obs = (250.0, 250.0, 250.0)
    tiny = h * 2.0 ** -23                      # rounds up to a whole cell at 21 fraction bits
    special = np.array([0.0, -0.0, 3 * h, 4 * h - tiny, 7.3 * h, L - 1e-9, L, -1e-9, -0.5 * L - 0.3,
                        L + 3.7, 2 * L - 1e-7, 3.5 * L, (n - 1) * h + 0.5 * h])
    grid = np.stack(np.meshgrid(special, special, special, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(11)
    gal = rng.uniform(0, L, (100_000, 3))
    ran = rng.uniform(0, L, (200_000, 3))
    r = B.Recon(n, L, 2.0, 0.7, 20.0, obs, periodic=True)
    # a position error e tilts the radial line of sight by e / |d|: images within 2 Mpc/h of the
    # observer (some combinations of the special values put one 0.3 Mpc/h away) are left to the
    # random shifts, which do not depend on it
    far = np.linalg.norm(np.mod(grid, L) - 250.0, axis=1) > 2.0
    assert far.sum() > 0.99 * len(grid)
    shifts = {}
    for path in (0, 1):
        r.set_option(B.OPT_DEPOSIT_PATH, path)
        r.set_option(B.OPT_SHIFT_PATH, path)
        # deposit: the special positions on top of a uniform catalogue
        both = np.concatenate([gal, grid])
        r.deposit(torch.from_numpy(both).cuda(), None, torch.from_numpy(ran).cuda(), None)
        rho_g = r.get_field(B.FIELD_RHO_G).cpu().numpy()
        assert abs(rho_g.astype(np.float64).sum() - len(both)) <= 1e-5 * len(both)
        # float32 sums in a run-dependent order: a node that collects m weights (a few hundred on
        # the corner node here) carries rounding of about sqrt(m) 2^-24 relative, so 1e-6 is within
        # reach of the rounding alone; 4e-6 is the bound
        assert rel_l2(rho_g, O.cic_deposit(both, None, n, L)) < 4e-6, path
        edge = rho_g - O.cic_deposit(gal, None, n, L)   # the special positions' share
        assert rel_l2(edge, O.cic_deposit(grid, None, n, L)) < 1e-5, path
        # shift: Psi of the uniform catalogues alone (the special positions would pile ~200 tracers
        # on the corner node, whose steep Psi would magnify the fixed-point position error),
        # interpolated at the special positions
        r.deposit(torch.from_numpy(gal).cuda(), None, torch.from_numpy(ran).cuda(), None)
        r.smooth()
        r.iterate(2, 0.0, 3)
        psi = r.get_psi().cpu().numpy().astype(np.float64)
        sg, pg = r.shift(torch.from_numpy(grid).cuda(), True, want_pos=True)
        sr = r.shift(torch.from_numpy(grid).cuda(), False)
        dg = O.shift_vectors(psi, grid, L, 0.7, obs, 0, True, periodic=True)
        dr = O.shift_vectors(psi, grid, L, 0.7, obs, 0, False)
        assert np.abs(sg.cpu().numpy() - dg)[far].max() <= SHIFT_TOL, path
        assert np.abs(sr.cpu().numpy() - dr).max() <= SHIFT_TOL, path
        assert np.abs(pg.cpu().numpy() - O.shifted_positions(grid, dg, L, True))[far].max() <= SHIFT_TOL, path
        shifts[path] = sr.cpu().numpy()
    assert np.abs(shifts[0] - shifts[1]).max() <= SHIFT_TOL
    r.close()


def test_smoothing_long_kernel_256(B):
    """A Gaussian wider than 64 taps on a mesh of at least 256 (the staged, unblocked convolution):
    delta of a uniform-density periodic box against the oracle's deposit, smoothing and delta."""
    n, L, R = 256, 500.0, 15.0                       # sigma = 7.7 cells: about 100 taps
    rng = np.random.default_rng(21)
    gal = rng.uniform(0, L, (400_000, 3))
    r = B.Recon(n, L, 2.0, 0.7, R, (250.0, 250.0, 250.0), periodic=True, uniform=True)
    r.deposit(torch.from_numpy(gal).cuda(), None, None, None)
    r.smooth()
    delta = r.get_field(B.FIELD_DELTA).cpu().numpy()
    r.close()
    rho = O.smooth(O.cic_deposit(gal, None, n, L), R, L)
    want = O.overdensity_uniform(rho, float(len(gal)))
    assert rel_l2(delta, want) < 1e-5


def test_empty_shift_catalogue(B):
    """A shift of no tracers (host or device, either path) returns (0, 3) and leaves the handle able
    to shift a real catalogue."""
    m = mocks.small_periodic(n_gal=20_000, n_ran=200_000, n_mesh=32)
    r = B.Recon.from_mock(m)
    n_it, rel, st = r.run(m.galaxies.pos, m.randoms.pos, start=0, tol=0.0, max_iter=2)
    assert n_it == 2
    for path in (0, 1):
        r.set_option(B.OPT_SHIFT_PATH, path)
        assert r.shift(np.zeros((0, 3)), True).shape == (0, 3)
        s, p = r.shift(torch.zeros((0, 3), dtype=torch.float64, device="cuda"), False, want_pos=True)
        assert tuple(s.shape) == (0, 3) and tuple(p.shape) == (0, 3)
    sg = r.shift(m.galaxies.pos, True)
    assert sg.shape == (len(m.galaxies.pos), 3) and np.isfinite(sg).all()
    r.close()


def test_cached_iteration_graph(B, periodic_mock, periodic_oracle):
    """recon_iterate keeps its instantiated graph: a repeated call relaunches it with the same result,
    and a changed start, tol or max_iter, or new parameters (recon_reconfigure), rebuilds it."""
    m = periodic_mock
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    r = B.Recon.from_mock(m)
    r.deposit(gal, None, ran, None)
    r.smooth()
    out = []
    for start, it in ((2, 6), (2, 6), (0, 6), (2, 4), (2, 6)):
        n_it, rel, st = r.iterate(start, 0.0, it)
        assert n_it == it
        out.append(r.get_psi().cpu().numpy())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[4])
    assert rel_l2(out[0], periodic_oracle[2]["psi"]) <= PSI_TOL
    assert rel_l2(out[2], periodic_oracle[0]["psi"]) <= PSI_TOL
    # new parameters through recon_reconfigure: the graph is rebuilt with the new b and f
    p = m.params()
    p2 = dict(p, b=2.5, f=0.6)
    prm = B.make_params(p2["n"], p2["L"], p2["b"], p2["f"], p2["R"], p2["observer"], p2["los_mode"], p2["periodic"],
                        p2["mask_frac"], p2["lognormal"], p2["uniform"])
    assert r.lib.recon_reconfigure(r.h, C.byref(prm)) == B.OK
    r.deposit(gal, None, ran, None)
    r.smooth()
    r.iterate(2, 0.0, 6)
    psi2 = r.get_psi().cpu().numpy()
    r.close()
    ref2 = O.reconstruct(p2, m.galaxies.pos, None, m.randoms.pos, None, start=O.START_FFTA, tol=0.0, max_iter=6)
    assert rel_l2(psi2, ref2["psi"]) <= PSI_TOL
