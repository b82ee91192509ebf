"""The synthetic input recipe (paper_1504_02591_gb300/mocks.py) against what it states: the
spectrum's normalisation and turnover, the survey window, tracer counts, the redshift-space shift
along each galaxy's line of sight, and the generator field's displacement convention."""
import numpy as np
import pytest

from paper_1504_02591_gb300 import mocks


def test_spectrum_is_normalised_to_unit_variance_at_R15():
    """sigma^2(R) = (1 / 2 pi^2) int P(k) exp(-k^2 R^2) k^2 dk = 1 at R = 15 Mpc/h (Gaussian window)."""
    integrate = pytest.importorskip("scipy.integrate")
    R = 15.0
    f = lambda k: mocks.power_spectrum(np.array([k]))[0] * np.exp(-(k * R) ** 2) * k * k / (2 * np.pi ** 2)
    var, _ = integrate.quad(f, 0.0, 5.0, limit=400, points=[0.01, 0.1, 0.3])
    assert var == pytest.approx(1.0, abs=1e-3)


def test_turnover_factor():
    """With k_turn the spectrum is multiplied by x / (1 + x), x = (k / k_turn)^2.5: one half at
    k_turn, and P grows as k^(-1.5 + 2.5) = k well below it."""
    k = np.array([0.02, 1e-4, 2e-4])
    p0, p1 = mocks.power_spectrum(k), mocks.power_spectrum(k, k_turn=0.02)
    assert p1[0] / p0[0] == pytest.approx(0.5, rel=1e-12)
    assert p1[2] / p1[1] == pytest.approx(2.0, rel=2e-5)
    assert mocks.power_spectrum(np.array([0.0]), k_turn=0.02)[0] == 0.0


def test_shell_survey_window_counts_and_line_of_sight():
    obs, r_lo, r_hi, sky = (0.0, 500.0, 500.0), 300.0, 480.0, 0.25
    m = mocks.shell_survey(1000.0, 32, 4000, 40000, 1.8, 0.7, 15.0, obs, (1.0, 0.0, 0.0), r_lo, r_hi, sky,
                           1, 2, 3, ng=32)
    assert len(m.galaxies.pos) == 4000 and len(m.randoms.pos) == 40000 and len(m.galaxies_real.pos) == 4000
    cos_min = 1.0 - 2.0 * sky          # a cap of solid angle 4 pi sky
    for p in (m.galaxies.pos, m.randoms.pos):
        d = p - np.asarray(obs)
        r = np.linalg.norm(d, axis=1)
        assert r.min() >= r_lo - 1e-9 and r.max() <= r_hi + 1e-9
        assert (d[:, 0] / r).min() >= cos_min - 1e-12
    # randoms fill the shell uniformly in volume: the median radius splits the shell volume in two
    r = np.linalg.norm(m.randoms.pos - np.asarray(obs), axis=1)
    r_half = np.cbrt(0.5 * (r_lo ** 3 + r_hi ** 3))
    assert abs(np.mean(r < r_half) - 0.5) < 0.01
    # the redshift-space shift runs along the line of sight through the real-space position
    x, s = m.galaxies_real.pos, m.galaxies.pos
    rh = (x - np.asarray(obs)) / np.linalg.norm(x - np.asarray(obs), axis=1, keepdims=True)
    assert np.abs(np.cross(s - x, rh)).max() < 1e-9 * max(1.0, np.abs(s - x).max())
    assert np.abs(s - x).max() > 0


def test_periodic_box_counts_and_wrap():
    m = mocks.periodic_box(800.0, 32, 5000, 20000, 2.0, 0.7, 15.0, (-400.0, 400.0, 400.0), 4, 5, 6, ng=32)
    assert len(m.galaxies.pos) == 5000 and len(m.randoms.pos) == 20000
    for p in (m.galaxies.pos, m.galaxies_real.pos, m.randoms.pos):
        assert p.min() >= 0.0 and p.max() < 800.0


def test_generator_displacement_is_the_zeldovich_field():
    """The generator's displacement is D(k) = i k delta(k) / k^2, so div D = -delta (first-order
    Lagrangian perturbation theory), checked mode by mode away from the Nyquist planes."""
    ng, L = 16, 600.0
    gf = mocks.gaussian_field(ng, L, 7)
    d = np.fft.rfftn(gf.delta.astype(np.float64))
    kf = 2 * np.pi / L
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    k = [kf * m[:, None, None], kf * m[None, :, None], kf * np.arange(ng // 2 + 1)[None, None, :]]
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    inner = (np.abs(m) < ng // 2)[:, None, None] & (np.abs(m) < ng // 2)[None, :, None] \
        & (np.arange(ng // 2 + 1) < ng // 2)[None, None, :] & (k2 > 0)
    for a in range(3):
        D = np.fft.rfftn(gf.disp[a].astype(np.float64))
        want = 1j * k[a] * d / np.where(k2 > 0, k2, 1.0)
        err = np.abs(D - want)[inner].max()
        assert err <= 1e-5 * np.abs(want)[inner].max()
