"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: a brute-force DFT, a closed form,
an explicit matrix solve, a finite-difference derivative, or an invariant.  Chosen so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import recon_oracle as O


def brute_rdft(a):
    """Definition of the 3-D forward DFT, sum_x a(x) exp(-2 pi i m.x / N), on the r2c half grid."""
    n = a.shape[0]
    idx = np.arange(n)
    E = np.exp(-2j * np.pi * np.outer(idx, idx) / n)          # E[m, x]
    full = np.einsum("ax,by,cz,xyz->abc", E, E, E, a)
    return full[:, :, : n // 2 + 1]


@pytest.mark.parametrize("n", [6, 8])
def test_fft_matches_brute_dft(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n, n))
    F = O.fft3(a)
    assert np.abs(F - brute_rdft(a)).max() <= 1e-12 * np.abs(F).max()
    assert np.abs(O.ifft3(F, n) - a).max() <= 1e-13 * np.abs(a).max()


def _mode(n, L, m, A=1.3, phase=0.0):
    x = np.arange(n) * (L / n)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"))
    k = 2 * np.pi * np.asarray(m, dtype=float) / L
    arg = (k[:, None, None, None] * X).sum(0) + phase
    return k, arg


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (1, 1, 0), (2, -1, 3), (3, 3, -2)])
def test_plane_wave_zeldovich(m):
    """delta = A cos(k.x)  =>  Psi = -(A/b) (k/k^2) sin(k.x) (Eq. Zeldovich, sign fixed by Eq. delta)."""
    n, L, A, b = 16, 500.0, 1.3, 1.9
    k, arg = _mode(n, L, m)
    delta = A * np.cos(arg)
    psi = O.zeldovich(delta / b, L)
    want = -(A / b) * (k[:, None, None, None] / (k @ k)) * np.sin(arg)[None]
    assert np.abs(psi - want).max() <= 1e-12 * np.abs(want).max()


def test_divergence_sign_against_finite_differences():
    """div Z[s] = -s, checked with a second-order central difference on a smooth field."""
    n, L = 64, 1000.0
    rng = np.random.default_rng(3)
    s = np.zeros((n, n, n))
    for _ in range(4):  # a few long-wavelength modes: FD error (kH)^2/6 <= 7e-3
        k, arg = _mode(n, L, rng.integers(-1, 2, 3) + np.array([1, 0, 0]))
        s += rng.standard_normal() * np.cos(arg + rng.uniform(0, 6))
    psi = O.zeldovich(s, L)
    H = L / n
    div = sum((np.roll(psi[j], -1, axis=j) - np.roll(psi[j], 1, axis=j)) / (2 * H) for j in range(3))
    assert np.abs(div + s).max() <= 1e-2 * np.abs(s).max()   # a sign error gives 2


def test_f_zero_converges_in_one_step():
    """f = 0: the source never changes, Psi_1 = Psi_0 = Z[delta/b] and rel = 0."""
    n, L = 16, 800.0
    delta = np.random.default_rng(0).standard_normal((n, n, n))
    rh = O.rhat_field(n, L, (1200.0, 400.0, 400.0), O.LOS_RADIAL)
    psi, rel, it = O.iterate(delta, 2.0, 0.0, L, rh, O.START_PLAIN, tol=1e-12, max_iter=5)
    assert it == 2 and max(rel) < 1e-15
    assert np.abs(psi - O.zeldovich(delta / 2.0, L)).max() < 1e-14 * np.abs(psi).max()


def _kaiser_parts(delta, b, L):
    n = delta.shape[0]
    _, kd, k2 = O.kgrid(n, L)
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1), 0.0)
    mu2 = kd[0] ** 2 * inv                   # (kd_x / k)^2, LOS along x
    return O.fft3(delta / b), mu2


@pytest.mark.parametrize("start", [O.START_PLAIN, O.START_APPROX1, O.START_FFTA])
def test_plane_parallel_iterates_closed_form(start):
    """Fixed LOS x: S_n = delta/b - beta mu^2 S_n-1, so every iterate has a closed form, and the
    limit is Kaiser Z[delta/b]/(1 + beta mu^2) (Eq. itpsi with the sign that matches Tables 2-3)."""
    n, L, b, f = 16, 600.0, 1.8, 0.7
    beta = f / b
    delta = np.random.default_rng(1).standard_normal((n, n, n))
    rh = O.rhat_field(n, L, (1.0, 0.0, 0.0), O.LOS_FIXED)
    _, rel, it, hist = O.iterate(delta, b, f, L, rh, start, tol=0.0, max_iter=8, return_all=True)
    D, mu2 = _kaiser_parts(delta, b, L)
    a = -beta * mu2
    c = O.start_coefficient(start, beta)
    # Psi_0 = Z[D] - c (Z[D].x) x  gives the radial source term (1-c) a D; S_0 = D + (1-c) a D
    S = D + (1 - c) * a * D
    for m in range(1, it + 1):
        want = np.stack([O.ifft3(ck, n) for ck in O.zeldovich_k(S, n, L)])
        got = hist[m]
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max(), m
        S = D + a * S
    kaiser = np.stack([O.ifft3(ck, n) for ck in O.zeldovich_k(D / (1 - a), n, L)])
    if start == O.START_PLAIN:
        # Psi_n = Psi_K [1 - (-beta mu^2)^(n+1)]
        for m in range(0, it + 1):
            want = np.stack([O.ifft3(ck, n) for ck in
                             O.zeldovich_k(D / (1 - a) * (1 - a ** (m + 1)), n, L)])
            assert np.abs(hist[m] - want).max() <= 1e-11 * np.abs(want).max()
    err = np.abs(hist[-1] - kaiser).max() / np.abs(kaiser).max()
    assert err < (beta ** (it + 1)) * 3


def test_approx1_exact_for_radial_mode():
    """A mode with k parallel to the LOS (mu = 1): Eq. approx1 is the exact Kaiser solution."""
    n, L, b, f = 16, 600.0, 2.0, 0.74
    k, arg = _mode(n, L, (2, 0, 0))
    delta = 0.8 * np.cos(arg)
    rh = O.rhat_field(n, L, (1.0, 0.0, 0.0), O.LOS_FIXED)
    beta = f / b
    psi_s = O.zeldovich(delta / b, L)
    psi0 = psi_s - O.start_coefficient(O.START_APPROX1, beta) * O.radial_projection(psi_s, rh)
    assert np.abs(psi0 - psi_s / (1 + beta)).max() < 1e-14
    psi, rel, it = O.iterate(delta, b, f, L, rh, O.START_APPROX1, tol=1e-13, max_iter=4)
    assert np.abs(psi - psi_s / (1 + beta)).max() < 1e-13 and it == 2


def _golden(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_ffta_coefficient_from_the_075_ratio():
    """Sec. 4.1: grad A = 0.75 curl B (the paper's measured x ratio, tests/golden/helmholtz_ratio.txt)
    and grad A + curl B = (Psi.r)r give grad A = (3/7)(Psi.r)r, so Eq. approx2's coefficient is
    (3/7)beta / (1 + (3/7)beta) = 3 beta/(7 + 3 beta)."""
    ratio = {row[0]: float(row[1]) for row in _golden("helmholtz_ratio.txt")}["x"]
    assert ratio == 0.75
    for beta in (0.2, 0.37, 0.4, 0.74):
        g = ratio / (1.0 + ratio)
        assert O.start_coefficient(O.START_FFTA, beta) == pytest.approx(g * beta / (1 + g * beta), rel=1e-15)
        assert O.start_coefficient(O.START_APPROX1, beta) == pytest.approx(beta / (1 + beta), rel=1e-15)


def _dft_matrix(n):
    idx = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(idx, idx) / n)


def test_radial_fixed_point_matches_dense_solve():
    """Radial LOS on 8^3: the converged iterate equals the solution of the linear system
    S - beta div_spec((Z[S].r)r) = delta/b assembled from explicit DFT matrices (no FFT library)."""
    n, L, b, f = 8, 400.0, 2.0, 0.6
    beta = f / b
    rng = np.random.default_rng(7)
    delta = rng.standard_normal((n, n, n))
    obs = (-150.0, 210.0, 130.0)
    rh = O.rhat_field(n, L, obs, O.LOS_RADIAL)
    E = _dft_matrix(n)
    F = np.kron(np.kron(E, E), E)                  # full 3-D DFT on flattened [x, y, z]
    Fi = np.conj(F) / n ** 3
    m = np.fft.fftfreq(n, 1.0 / n)
    kk = 2 * np.pi * m / L
    kdd = np.where(np.abs(m) == n // 2, 0.0, kk)
    KX, KY, KZ = np.meshgrid(kk, kk, kk, indexing="ij")
    DX, DY, DZ = np.meshgrid(kdd, kdd, kdd, indexing="ij")
    k2 = (KX ** 2 + KY ** 2 + KZ ** 2).ravel()
    inv = np.where(k2 > 0, 1 / np.where(k2 > 0, k2, 1), 0.0)
    kd = [DX.ravel(), DY.ravel(), DZ.ravel()]
    Z = [np.real(Fi @ np.diag(1j * kd[j] * inv) @ F) for j in range(3)]        # S -> Psi_j
    Dv = [np.real(Fi @ np.diag(1j * kd[j]) @ F) for j in range(3)]             # P_j -> div part
    R = [rh[j].ravel() for j in range(3)]
    proj = sum(np.diag(R[j]) @ Z[j] for j in range(3))                          # S -> Psi.r
    DP = sum(Dv[j] @ np.diag(R[j]) @ proj for j in range(3))                    # S -> div((Psi.r)r)
    A = np.eye(n ** 3) - beta * DP
    S = np.linalg.solve(A, (delta / b).ravel())
    want = np.stack([(Z[j] @ S).reshape(n, n, n) for j in range(3)])
    psi, rel, it = O.iterate(delta, b, f, L, rh, O.START_FFTA, tol=1e-14, max_iter=200)
    assert np.abs(psi - want).max() <= 1e-10 * np.abs(want).max()


def test_distant_observer_tends_to_kaiser():
    """A radial LOS from an observer far along -x approaches the plane-parallel Kaiser solution."""
    n, L, b, f = 16, 500.0, 2.0, 0.74
    delta = np.random.default_rng(5).standard_normal((n, n, n))
    rh = O.rhat_field(n, L, (-1e7, 250.0, 250.0), O.LOS_RADIAL)
    psi, _, _ = O.iterate(delta, b, f, L, rh, O.START_PLAIN, tol=1e-12, max_iter=100)
    D, mu2 = _kaiser_parts(delta, b, L)
    kaiser = np.stack([O.ifft3(ck, n) for ck in O.zeldovich_k(D / (1 + f / b * mu2), n, L)])
    assert np.abs(psi - kaiser).max() <= 1e-4 * np.abs(kaiser).max()


def test_cic_mass_and_node_and_adjoint():
    n, L = 12, 300.0
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, L, (5000, 3))
    w = rng.uniform(0.5, 2.0, 5000)
    rho = O.cic_deposit(pos, w, n, L)
    assert abs(rho.sum() - w.sum()) <= 1e-12 * w.sum()
    # a particle exactly on a node deposits its whole weight on that node
    node = np.array([[3, 7, 11]]) * (L / n)
    r1 = O.cic_deposit(node, np.array([2.5]), n, L)
    assert r1[3, 7, 11] == 2.5 and np.count_nonzero(r1) == 1
    # wrap: a particle at u = n - 0.25 shares with node 0
    r2 = O.cic_deposit(np.array([[L - 0.25 * L / n, 0.0, 0.0]]), None, n, L)
    assert r2[n - 1, 0, 0] == pytest.approx(0.25) and r2[0, 0, 0] == pytest.approx(0.75)
    # adjointness <deposit(w), F> = sum_p w_p gather(F)(x_p)
    F = rng.standard_normal((n, n, n))
    assert (rho * F).sum() == pytest.approx((w * O.cic_gather(F, pos, L)).sum(), rel=1e-12)


def test_cic_gathers_linear_field_exactly():
    n, L = 16, 160.0
    x = np.arange(n) * (L / n)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"))
    a, g = 0.3, np.array([0.7, -1.1, 0.4])
    F = a + (g[:, None, None, None] * X).sum(0)
    pos = np.random.default_rng(2).uniform(0, L - L / n, (2000, 3))   # away from the wrap
    assert np.abs(O.cic_gather(F, pos, L) - (a + pos @ g)).max() < 1e-12


def test_smoothing_single_mode():
    n, L, R = 32, 640.0, 15.0
    k, arg = _mode(n, L, (2, 1, 0))
    out = O.smooth(np.cos(arg), R, L)
    assert np.abs(out - np.exp(-0.5 * (k @ k) * R * R) * np.cos(arg)).max() < 1e-13


def test_lognormal_small_delta_and_mean():
    rng = np.random.default_rng(4)
    d = 1e-3 * rng.standard_normal((8, 8, 8))
    ld, C = O.lognormal(d)
    want = d - d * d / 2 + d ** 3 / 3 - d ** 4 / 4     # Taylor series; next term ~ 2e-13
    want = want - want.mean()
    assert np.abs(ld - want).max() < 1e-12
    assert abs(ld.mean()) < 1e-17 and C == pytest.approx(-np.log(1 + d).mean(), rel=1e-12)


def test_overdensity_zero_when_galaxies_trace_randoms():
    rng = np.random.default_rng(8)
    rr = rng.uniform(0.1, 2.0, (8, 8, 8))
    rr[0, 0, :4] = 0.0
    d, mask, alpha, thr = O.overdensity_randoms(3.0 * rr, rr, 30.0, 10.0, 0.01, 500)
    assert alpha == 3.0 and not mask[0, 0, 0] and mask[4, 4, 4]
    assert np.abs(d).max() < 1e-15
    assert thr == pytest.approx(0.01 * 10.0 / 500)


def test_shift_periodic_images():
    """Periodic box: moving a tracer by whole box lengths changes neither its interpolated Psi nor,
    with the image reading, its line of sight, so the shifts are identical; without it the radial
    LOS of an out-of-box image differs."""
    n, L, f = 8, 200.0, 0.74
    rng = np.random.default_rng(10)
    psi = rng.standard_normal((3, n, n, n))
    pos = rng.uniform(0, L, (200, 3))
    k = rng.integers(-3, 4, (200, 3)).astype(np.float64)
    k[0] = (1, 0, 0)
    img = pos + L * k
    obs = (100.0, 100.0, 100.0)
    d0 = O.shift_vectors(psi, pos, L, f, obs, O.LOS_RADIAL, True, periodic=True)
    d1 = O.shift_vectors(psi, img, L, f, obs, O.LOS_RADIAL, True, periodic=True)
    assert np.abs(d0 - d1).max() < 1e-9
    d2 = O.shift_vectors(psi, img, L, f, obs, O.LOS_RADIAL, True, periodic=False)
    assert np.abs(d0 - d2).max() > 1e-3
    r0 = O.shift_vectors(psi, pos, L, f, obs, O.LOS_RADIAL, False)
    r1 = O.shift_vectors(psi, img, L, f, obs, O.LOS_RADIAL, False)
    assert np.abs(r0 - r1).max() < 1e-9


def test_shift_decomposition():
    """Galaxy shift: along the LOS -(1+f)(Psi.r); across it -Psi_perp.  Randoms: -Psi."""
    n, L, f = 8, 200.0, 0.74
    rng = np.random.default_rng(9)
    psi = rng.standard_normal((3, n, n, n))
    pos = rng.uniform(0, L, (300, 3))
    obs = (-100.0, 50.0, 20.0)
    p = O.cic_gather(psi, pos, L)
    rh = O.particle_rhat(pos, obs, O.LOS_RADIAL)
    dg = O.shift_vectors(psi, pos, L, f, obs, O.LOS_RADIAL, True)
    dr = O.shift_vectors(psi, pos, L, f, obs, O.LOS_RADIAL, False)
    par = (p * rh).sum(1)
    assert np.abs((dg * rh).sum(1) + (1 + f) * par).max() < 1e-12
    perp_g = dg - (dg * rh).sum(1)[:, None] * rh
    perp_p = p - par[:, None] * rh
    assert np.abs(perp_g + perp_p).max() < 1e-12
    assert np.abs(dr + p).max() == 0.0
    assert np.allclose(np.linalg.norm(rh, axis=1), 1.0)


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 3, 0), (2, -1, 1)])
def test_divergence_of_a_plane_wave(m):
    """div of v = a sin(k.x) (constant vector a) is (a.k) cos(k.x), exactly for a mode on the mesh."""
    n, L = 16, 300.0
    k, arg = _mode(n, L, m)
    a = np.array([0.7, -1.1, 0.4])
    v = a[:, None, None, None] * np.sin(arg)[None]
    got = O.ifft3(O.divergence(v, L), n)
    assert np.abs(got - (a @ k) * np.cos(arg)).max() < 1e-12


def test_overdensity_uniform_single_mode():
    """rho = c (1 + e cos(k.x)) has mean c, so delta = e cos(k.x) exactly."""
    n = 8
    _, arg = _mode(n, 100.0, (1, 2, 0))
    c, e = 2.5, 0.3
    rho = c * (1.0 + e * np.cos(arg))
    d = O.overdensity_uniform(rho, rho.sum())
    assert np.abs(d - e * np.cos(arg)).max() < 1e-14
    d2 = O.overdensity_uniform(rho, 2.0 * rho.sum())           # twice the mean: (1 + e cos)/2 - 1
    assert np.abs(d2 - (0.5 * (1.0 + e * np.cos(arg)) - 1.0)).max() < 1e-14


def test_shifted_positions_wrap_only_when_periodic():
    L = 100.0
    pos = np.array([[99.9, 0.05, 50.0]])
    d = np.array([[0.3, -0.1, 0.0]])
    assert np.allclose(O.shifted_positions(pos, d, L, True), [[0.2, 99.95, 50.0]], atol=1e-12)
    assert np.allclose(O.shifted_positions(pos, d, L, False), [[100.2, -0.05, 50.0]], atol=1e-12)


def test_reconstruct_galaxies_tracing_randoms_is_still():
    """Randoms that are the galaxies three times over: alpha = 1/3 and delta = 0 in the mask, so the
    whole pipeline returns Psi = 0 and zero shifts (an inverted alpha, a field smoothed twice or not
    at all, or a mask applied to one side only would not)."""
    rng = np.random.default_rng(12)
    n, L = 16, 400.0
    gal = rng.uniform(100.0, 300.0, (3000, 3))
    ran = np.concatenate([gal, gal, gal])
    p = dict(n=n, L=L, b=2.0, f=0.7, R=30.0, los_mode=O.LOS_RADIAL, observer=(0.0, 200.0, 200.0),
             periodic=False, mask_frac=0.01, lognormal=False, uniform=False)
    out = O.reconstruct(p, gal, None, ran, None, start=O.START_FFTA, tol=0.0, max_iter=3)
    assert out["alpha"] == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert out["mask"].any() and not out["mask"].all()
    assert np.abs(out["delta"]).max() < 1e-12
    assert np.abs(out["psi"]).max() < 1e-12
    assert np.abs(out["shift_g"]).max() < 1e-12 and np.abs(out["shift_r"]).max() < 1e-12


def test_rhat_nodes_sit_at_i_times_H():
    """Sec. 3.1: the line of sight is the unit vector from the observer to the point.  With the
    observer placed exactly on node (i, j, k) (observer = (i, j, k) H), the node-centred field must
    vanish on that node and be the axis unit vectors on its six neighbours and (1, 1, 0)/sqrt(2) on a
    diagonal one; a grid offset by any fraction of a cell (nodes at (i + 1/2) H, say) would give a
    non-zero vector at the observer's node and tilted vectors at the neighbours."""
    n, L = 16, 320.0
    H = L / n
    i, j, k = 5, 9, 12
    rh = O.rhat_field(n, L, (i * H, j * H, k * H), O.LOS_RADIAL)
    assert np.array_equal(rh[:, i, j, k], [0.0, 0.0, 0.0])
    for axis in range(3):
        for step in (-1, 1):
            node = [i, j, k]
            node[axis] += step
            want = np.zeros(3)
            want[axis] = step
            assert np.abs(rh[:, node[0], node[1], node[2]] - want).max() < 1e-15
    s = 1.0 / np.sqrt(2.0)
    assert np.abs(rh[:, i + 1, j + 1, k] - [s, s, 0.0]).max() < 1e-15
    assert np.abs(rh[:, i, j - 3, k - 4] - [0.0, -0.6, -0.8]).max() < 1e-15   # a 3-4-5 triangle
    # the field is a unit vector everywhere else
    r = np.sqrt((rh * rh).sum(0))
    r[i, j, k] = 1.0
    assert np.abs(r - 1.0).max() < 1e-14


def test_mask_threshold_counts_touched_nodes_by_hand():
    """Sec. 3.2 survey mask reading: the threshold is mask_frac x sum w_r / (nodes that received
    random mass).  Hand-built randoms: one on a node (touches 1 node), one at a cell centre
    (touches 8), one more inside that same cell (the same 8 nodes) and one halfway along an x edge
    of another cell (touches the edge's 2 end nodes): 1 + 8 + 2 = 11 nodes, total weight 5."""
    n, L = 16, 160.0            # H = 10
    ran = np.array([[20.0, 30.0, 40.0],     # node (2, 3, 4): 1 node
                    [105.0, 105.0, 105.0],  # centre of cell (10, 10, 10): nodes 10..11 ^3, 8 nodes
                    [102.0, 107.0, 103.5],  # inside the same cell: the same 8 nodes
                    [55.0, 150.0, 0.0]])    # on the x edge of cell (5, 15, 0): nodes (5|6, 15, 0)
    wr = np.array([1.0, 1.0, 1.0, 2.0])
    gal = np.array([[50.0, 50.0, 50.0]])
    p = dict(n=n, L=L, b=2.0, f=0.7, R=10.0, los_mode=O.LOS_RADIAL, observer=(0.0, 80.0, 80.0),
             periodic=False, mask_frac=0.01, lognormal=False, uniform=False)
    out = O.reconstruct(p, gal, None, ran, wr, start=O.START_PLAIN, tol=0.0, max_iter=1, shift=False)
    assert np.count_nonzero(out["rho_r"] > 0) == 11
    assert out["threshold"] == pytest.approx(0.01 * 5.0 / 11.0, rel=1e-15)
    assert out["alpha"] == pytest.approx(1.0 / 5.0, rel=1e-15)


def test_lognormal_floor_branch():
    """Eq. logdelta with 1 + delta floored at 1e-6: delta = -1 and delta = -3 both give
    ln(1e-6) = -6 ln 10, and C = -<ln(max(1 + delta, 1e-6))>."""
    e = np.e
    delta = np.array([-1.0, -3.0, e - 1.0, e * e - 1.0])
    ln_floor = -6.0 * np.log(10.0)
    raw = np.array([ln_floor, ln_floor, 1.0, 2.0])
    out, C = O.lognormal(delta)
    assert C == pytest.approx(-raw.mean(), rel=1e-14)
    assert np.abs(out - (raw - raw.mean())).max() < 1e-13
    # just above the floor the logarithm is not clipped
    d2 = np.array([-1.0 + 2e-6, 0.0])
    out2, C2 = O.lognormal(d2)
    assert out2[0] - out2[1] == pytest.approx(np.log(2e-6), rel=1e-9)


def test_ratio_stats_outlier_rule_by_hand():
    """Tables 1-3: ratios above 3 or below -1 are cut; a zero denominator is an outlier."""
    num = np.array([1.0, 2.0, 9.0, -4.0, 1.5, 0.5, 3.0])
    den = np.array([1.0, 1.0, 1.0, 2.0, 0.0, 1.0, 1.0])      # ratios 1, 2, 9 (cut), -2 (cut), -, 0.5, 3
    mean, std, out, kept = O.ratio_stats(num, den)
    r = np.array([1.0, 2.0, 0.5, 3.0])
    assert kept == 4 and out == pytest.approx(3.0 / 7.0)
    assert mean == pytest.approx(1.625) and std == pytest.approx(np.sqrt(((r - 1.625) ** 2).mean()))


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (1, 1, 0), (2, -1, 3), (1, 2, 2)])
def test_helmholtz_split_of_a_single_mode(m):
    """Eq. irrotational / Eq. solenoidal on Psi_x = cos(k.x): grad A = (k_j k_x / k^2) cos(k.x) and
    curl B = ((k_y^2 + k_z^2), -k_y k_x, -k_z k_x) cos(k.x) / k^2, so the x-ratio of the two is
    k_x^2 / (k_y^2 + k_z^2) and the y, z ratios are -1 wherever they are defined; grad A is curl-free,
    curl B divergence-free, and the two add up to (Psi.x) x."""
    n, L = 16, 400.0
    k, arg = _mode(n, L, m)
    psi = np.zeros((3, n, n, n))
    psi[0] = np.cos(arg)
    psi[1] = 0.7 * np.sin(arg)            # components other than x play no part
    ga, cb = O.helmholtz_x(psi, L)
    k2 = k @ k
    c = np.cos(arg)
    assert np.abs(ga - (k[:, None, None, None] * k[0] / k2) * c).max() < 1e-12
    want_cb = np.stack([(k[1] ** 2 + k[2] ** 2) / k2 * c, -k[1] * k[0] / k2 * c, -k[2] * k[0] / k2 * c])
    assert np.abs(cb - want_cb).max() < 1e-12
    assert np.abs(ga + cb - np.stack([psi[0], 0 * c, 0 * c])).max() < 1e-12
    # curl of grad A and divergence of curl B vanish (spectral derivatives)
    _, kd, _ = O.kgrid(n, L)
    GA = [O.fft3(g) for g in ga]
    curl = [kd[1] * GA[2] - kd[2] * GA[1], kd[2] * GA[0] - kd[0] * GA[2], kd[0] * GA[1] - kd[1] * GA[0]]
    assert max(np.abs(cc).max() for cc in curl) < 1e-9
    div_cb = sum(kd[j] * O.fft3(cb[j]) for j in range(3))
    assert np.abs(div_cb).max() < 1e-9


def test_radial_ratio_uses_each_particles_line_of_sight():
    """Eq. ratio at particles: constant fields Psi_real = (2, 0, 0), Psi_est = (4, 3, 0) seen from an
    observer at the box centre: a particle along +x gives 2/4, one along +y gives 0/3, one along
    the (1, 1, 0) diagonal gives (2/sqrt2)/(7/sqrt2) = 2/7."""
    n, L = 8, 80.0
    real = np.zeros((3, n, n, n))
    est = np.zeros((3, n, n, n))
    real[0] = 2.0
    est[0], est[1] = 4.0, 3.0
    obs = (40.0, 40.0, 40.0)
    pos = np.array([[70.0, 40.0, 40.0], [40.0, 55.0, 40.0], [50.0, 50.0, 40.0]])
    mean, std, out, kept = O.radial_ratio(real, est, pos, L, obs, O.LOS_RADIAL)
    r = np.array([0.5, 0.0, 2.0 / 7.0])
    assert kept == 3 and out == 0.0
    assert mean == pytest.approx(r.mean(), rel=1e-12) and std == pytest.approx(r.std(), rel=1e-12)


def test_ngp_deposit_by_hand():
    """Sec. 3 NGP: a particle goes to its nearest node; halfway between nodes it goes up; periodic."""
    n, L = 8, 80.0                                  # H = 10
    pos = np.array([[14.9, 25.0, 0.0], [15.0, 24.9, 79.0], [79.9, 0.1, 44.0]])
    rho = O.ngp_deposit(pos, np.array([1.0, 2.0, 4.0]), n, L)
    assert rho[1, 3, 0] == 1.0            # (1.49, 2.5, 0) -> (1, 3, 0)
    assert rho[2, 2, 0] == 2.0            # (1.5, 2.49, 7.9) -> (2, 2, 8 = 0)
    assert rho[0, 0, 4] == 4.0            # (7.99, 0.01, 4.4) -> (8 = 0, 0, 4)
    assert rho.sum() == 7.0 and np.count_nonzero(rho) == 3


def test_radial_nbar_and_fkp_weights():
    """n(r) of a uniform shell catalogue is its number over the shell's volume; FKP weights
    1/(1 + n P0) (Sec. 3.2) by hand, with n = 0 outside the shells."""
    obs = np.array([100.0, 100.0, 100.0])
    # 3 particles at r = 10, 2 at r = 25, one at r = 40 (outside the shells [0, 20) and [20, 30))
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, -1], [0.6, 0.8, 0], [0, -0.6, 0.8], [1, 0, 0]], dtype=float)
    rr = np.array([10.0, 10.0, 10.0, 25.0, 25.0, 40.0])
    pos = obs + dirs * rr[:, None]
    edges = [0.0, 20.0, 30.0]
    sky = 2.0
    nbar = O.radial_nbar(pos, obs, edges, sky)
    want = np.array([3.0 / (sky * 20.0 ** 3 / 3.0), 2.0 / (sky * (30.0 ** 3 - 20.0 ** 3) / 3.0)])
    assert np.allclose(nbar, want, rtol=1e-14)
    w = O.fkp_weights(pos, obs, edges, nbar, P0=20000.0)
    assert np.allclose(w, [1 / (1 + want[0] * 2e4)] * 3 + [1 / (1 + want[1] * 2e4)] * 2 + [1.0], rtol=1e-14)


def _dst_mode(n, m):
    """Discrete sine mode sin(pi m_a (i_a + 1) / (n + 1)) per axis: zero just outside the mesh."""
    i = np.arange(n) + 1.0
    s = [np.sin(np.pi * mm * i / (n + 1)) for mm in m]
    return s[0][:, None, None] * s[1][None, :, None] * s[2][None, None, :]


def test_fd_operator_eigenmodes():
    """Sec. 2.1 stencils with phi = 0 outside the mesh: a discrete sine mode is an eigenvector of
    the 7-point Laplacian with eigenvalue sum_a (2 cos(pi m_a / (n + 1)) - 2) / g^2, and for a fixed
    line of sight along x the line-of-sight term adds beta (2 cos(pi m_x / (n + 1)) - 2) / g^2."""
    n, L = 12, 300.0
    g = L / n
    m = (2, 3, 5)
    phi = _dst_mode(n, m)
    lam = [(2.0 * np.cos(np.pi * mm / (n + 1)) - 2.0) / g ** 2 for mm in m]
    assert np.abs(O.fd_operator(phi, L, 0.0, (1, 0, 0), O.LOS_FIXED) - sum(lam) * phi).max() < 1e-12
    beta = 0.4
    got = O.fd_operator(phi, L, beta, (1, 0, 0), O.LOS_FIXED)
    assert np.abs(got - (sum(lam) + beta * lam[0]) * phi).max() < 1e-12


def test_fd_fixed_los_stencil_is_symmetric_and_radial_is_second_order():
    """The fixed-LOS stencil (central second differences) is symmetric; the radial one, with its
    (2/r) d/dr term, approximates div((grad phi . r) r) of a smooth blob to second order in g."""
    rng = np.random.default_rng(4)
    n, L = 10, 200.0
    a, b = rng.standard_normal((2, n, n, n))
    u = (0.3, -0.5, 0.81)
    Aa, Ab = (O.fd_operator(v, L, 0.7, u, O.LOS_FIXED) for v in (a, b))
    assert (b * Aa).sum() == pytest.approx((a * Ab).sum(), rel=1e-12)
    obs = np.array([-150.0, 80.0, 120.0])
    errs = []
    for n in (32, 64):
        L = 200.0
        g = L / n
        x = np.arange(n) * g
        X = np.stack(np.meshgrid(x, x, x, indexing="ij"))
        c, s2 = np.array([100.0, 100.0, 100.0]), 18.0 ** 2
        dX = X - c[:, None, None, None]
        phi = np.exp(-(dX ** 2).sum(0) / (2 * s2))
        grad = -dX / s2 * phi
        hess = [[(dX[i] * dX[j] / s2 ** 2 - (i == j) / s2) * phi for j in range(3)] for i in range(3)]
        d = X - obs[:, None, None, None]
        r = np.sqrt((d ** 2).sum(0))
        rh = d / r
        exact = sum(rh[i] * rh[j] * hess[i][j] for i in range(3) for j in range(3)) + \
            (2.0 / r) * sum(rh[i] * grad[i] for i in range(3))
        fd = O.fd_operator(phi, L, 1.0, obs, O.LOS_RADIAL) - O.fd_operator(phi, L, 0.0, obs, O.LOS_RADIAL)
        errs.append(np.abs(fd - exact).max() / np.abs(exact).max())
    assert errs[1] < 1e-2 and errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)


def test_fd_solve_matches_sine_transform_solution():
    """f = 0 and a fixed line of sight along x: the operator is diagonal in the discrete sine basis,
    so the exact solution is a sine transform; the GMRES solve (with its FFT preconditioner for the
    periodic Laplacian) must reproduce it, and Psi = -grad phi by central differences."""
    from scipy.fft import dstn, idstn
    n, L, b = 24, 480.0, 2.0
    g = L / n
    rng = np.random.default_rng(9)
    delta = O.smooth(rng.standard_normal((n, n, n)), 40.0, L)
    m = np.arange(1, n + 1)
    lam1 = (2.0 * np.cos(np.pi * m / (n + 1)) - 2.0) / g ** 2
    lap = lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]
    for f in (0.0, 0.8):
        eig = lap + (f / b) * lam1[:, None, None]
        want = idstn(dstn(delta / b, type=1) / eig, type=1)
        psi, phi, it, res = O.fd_solve(delta, b, f, L, (1.0, 0.0, 0.0), O.LOS_FIXED, tol=1e-12)
        assert np.abs(phi - want).max() < 1e-9 * np.abs(want).max()
        ppad = np.pad(want, 1)
        gx = -(ppad[2:, 1:-1, 1:-1] - ppad[:-2, 1:-1, 1:-1]) / (2 * g)
        assert np.abs(psi[0] - gx).max() < 1e-9 * np.abs(gx).max()


def test_convergence_rule_reproduces_the_papers_tables():
    """Sec. 5.2, Tables 2 and 3 (tests/golden/iteration_tables.txt): the rule applied to the
    paper's printed mean ratios gives the iteration counts its captions state.  The strict relative
    reading (each change below 1% of the previous mean) does not: Table 2's uncorrected run changes
    by 0.01 from 0.99, which is 1.01%, so it would converge at 5, not 4."""
    rows = _golden("iteration_tables.txt")
    means, stated = {}, {}
    for row in rows:
        if row[0] == "converged":
            stated[(row[1], row[2])] = int(row[3])
        else:
            means.setdefault((row[0], row[1]), []).append((int(row[2]), float(row[3])))
    assert set(stated) == set(means) and len(stated) == 4
    for key, seq in means.items():
        seq = [m for _, m in sorted(seq)]
        assert O.converged_at(seq) == stated[key], key
    # the paper's pattern: from the uncorrected start the mean starts low and oscillates about 1
    for t in ("table2", "table3"):
        m = [x for _, x in sorted(means[(t, "plain")])]
        assert m[0] < 1 and all((m[k] - 1) * (m[k + 1] - 1) < 0 for k in range(3))
    plain2 = [x for _, x in sorted(means[("table2", "plain")])]
    strict = next(n for n in range(len(plain2))
                  if all(abs(plain2[k + 1] - plain2[k]) < 0.01 * abs(plain2[k]) for k in range(n, len(plain2) - 1)))
    assert strict == 5


def test_nyquist_mode_takes_the_mean_of_its_two_aliases():
    """On the mesh, a mode with the Nyquist index along x, m = (N/2, 1, 0), is the same field as its
    alias (-N/2, 1, 0), and Eq. Zeldovich gives the two opposite x components.  The real answer is
    their mean (the reading of the Nyquist index: derivative wavenumber 0 along x there, k^2 the
    full |k|^2): Psi_x = 0, Psi_y = -(A/b) (k_y/k^2) sin(k.x) with k^2 = k_N^2 + k_y^2."""
    n, L, A, b = 16, 400.0, 0.9, 2.1
    k, arg = _mode(n, L, (n // 2, 1, 0))
    delta = A * np.cos(arg)
    psi = O.zeldovich(delta / b, L)
    k_alias = k * np.array([-1.0, 1.0, 1.0])
    arg_alias = _mode(n, L, (-n // 2, 1, 0))[1]
    assert np.abs(np.cos(arg_alias) - np.cos(arg)).max() < 1e-12      # the same field on the nodes
    want = -(A / b) * 0.5 * (k[:, None, None, None] * np.sin(arg)[None]
                             + k_alias[:, None, None, None] * np.sin(arg_alias)[None]) / (k @ k)
    assert np.abs(psi[0]).max() < 1e-13
    assert np.abs(psi - want).max() <= 1e-12 * np.abs(want).max()
    assert np.abs(want[1]).max() > 0.1 * A / b / np.sqrt(k @ k)      # the y component is not trivial


def test_divergence_of_a_nyquist_mode():
    """div of v = a sin(k.x) with the Nyquist index along x: the field equals its (-N/2, 1, 0) alias,
    whose divergences (a.k) cos(k.x) differ in the x term, so the answer is their mean,
    a_y k_y cos(k.x)."""
    n, L = 16, 300.0
    k, arg = _mode(n, L, (n // 2, 1, 0))
    a = np.array([0.7, -1.1, 0.4])
    v = a[:, None, None, None] * np.sin(arg)[None]
    got = O.ifft3(O.divergence(v, L), n)
    assert np.abs(got - a[1] * k[1] * np.cos(arg)).max() < 1e-12


def test_updates_are_curl_free():
    """Every update of Eq. iterative is Psi = Z[S] = i k S / k^2, a gradient: k x Psi(k) = 0 (with the
    derivative wavenumbers, Nyquist index zero), also for a radial line of sight where (Psi.r)r itself
    has a curl; and its divergence is -S."""
    n, L, b, f = 12, 300.0, 1.7, 0.8
    rng = np.random.default_rng(21)
    delta = rng.standard_normal((n, n, n))
    rh = O.rhat_field(n, L, (-150.0, 120.0, 170.0), O.LOS_RADIAL)
    psi0, _ = O.start_estimate(delta, b, f, L, rh, O.START_FFTA)
    psi1 = O.update(psi0, delta, b, f, L, rh)
    _, kd, _ = O.kgrid(n, L)
    P = [O.fft3(psi1[j]) for j in range(3)]
    scale = max(np.abs(p).max() for p in P)
    for a, c in ((1, 2), (2, 0), (0, 1)):
        assert np.abs(kd[a] * P[c] - kd[c] * P[a]).max() <= 1e-12 * scale * np.abs(kd[0]).max()
    proj = O.radial_projection(psi0, rh)
    Q = [O.fft3(proj[j]) for j in range(3)]
    curl_proj = max(np.abs(kd[a] * Q[c] - kd[c] * Q[a]).max() for a, c in ((1, 2), (2, 0), (0, 1)))
    assert curl_proj > 1e-3 * max(np.abs(q).max() for q in Q) * np.abs(kd[0]).max()
    S_k = O.fft3(delta / b) + (f / b) * O.divergence(proj, L)
    S_k[0, 0, 0] = 0.0
    div = sum(1j * kd[j] * P[j] for j in range(3))
    k, _, k2 = O.kgrid(n, L)
    keep = (k2 > 0) & (kd[0] == k[0]) & (kd[1] == k[1]) & (kd[2] == k[2])   # no Nyquist index
    assert keep.sum() > 0.5 * keep.size
    assert np.abs(div + S_k)[keep].max() <= 1e-12 * np.abs(S_k).max()
