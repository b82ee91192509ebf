"""FP64 CPU oracle for iterative Fourier-space reconstruction (Burden, Percival & Howlett 2015).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct reference that the CUDA path
is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline``, ``--cpu-full`` and the ``--impl reference`` arm) may import it.  The product path (``paper_1504_02591_gb300``) never imports, calls or
links it, and it shares no code with the CUDA kernels.

Everything is float64 numpy.  The 3-D FFT is ``scipy.fft.rfftn`` / ``irfftn`` used as a library
primitive (forward e^{-ik.x} unnormalised, inverse with 1/N^3), run on ``FFT_WORKERS`` host threads
(all cores by default; a caller may set it, e.g. to 1 for a single-core timing); the test suite pins
it against a brute-force DFT.  There is no blocking, fusion or reordering beyond what the paper's
equations state.

Conventions (readings of the paper where it is silent or inconsistent, stated here once):

* Grid: nodes at x_i = i*H, i = 0..N-1 per axis, H = L/N, periodic.  Arrays are indexed [ix, iy, iz].
* k_j = 2 pi m_j / L with m_j in {0..N/2-1, -N/2..-1}.  The derivative wavenumber kd_j equals k_j
  except at the Nyquist index m_j = N/2 where it is 0 (keeps real fields real); k^2 uses the full k.
* Zel'dovich operator (Eq. Zeldovich): Z[s](k) = i kd s(k) / k^2, with Z[s](k=0) = 0, so that
  div Z[s] = -s (Eq. delta) for every mode whose kd = k.
* The solved equation is Eq. Nusser with the redshift-space coefficient read as beta = f/b:
  div Psi + beta div((Psi.r)r) = -delta/b.  With S = delta/b + beta div((Psi.r)r) this is Psi = Z[S].
  The sign is fixed by the plane-parallel Kaiser limit S = (delta/b)/(1 + beta mu^2).
* Smoothing kernel exp(-k^2 R^2 / 2) (the printed "-ik^2R^2/2" of Sec. 3.1 read as a real Gaussian).
* CIC (cloud-in-cell) mass assignment on the nodes, periodic wrap; the paper bins with NGP (Sec. 3).
* Tracers outside a periodic box: a position stands for its image in [0, L); the mesh wraps it and a
  galaxy's radial line of sight runs from the observer to that image (the paper is silent).
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as _sfft

LOS_RADIAL = 0
LOS_FIXED = 1

START_PLAIN = 0      # Psi_red,FFT: no RSD correction (Sec. 5.2, first starting point)
START_APPROX1 = 1    # Eq. approx1: irrotational approximation, coefficient beta/(1+beta)
START_FFTA = 2       # Eq. approx2: 0.75-ratio approximation, coefficient 3 beta/(7+3 beta)

LOG_FLOOR = 1e-6     # floor on 1+delta before the logarithm of Eq. logdelta

FFT_WORKERS = os.cpu_count() or 1   # host threads of the library FFT (results do not depend on it)


# --------------------------------------------------------------------------------------------
# Fourier grid
# --------------------------------------------------------------------------------------------
def axis_wavenumbers(n: int, L: float, half: bool = False):
    """Wavenumbers of one axis: (k, kd).  ``half`` gives the r2c axis (m = 0..n/2)."""
    if half:
        m = np.arange(n // 2 + 1, dtype=np.float64)
    else:
        m = np.fft.fftfreq(n, d=1.0 / n)
    k = 2.0 * np.pi * m / L
    kd = k.copy()
    if n % 2 == 0:
        kd[np.abs(m) == n // 2] = 0.0
    return k, kd


def kgrid(n: int, L: float):
    """Broadcastable (kx, ky, kz), (kdx, kdy, kdz) and k^2 on the rfftn grid (n, n, n/2+1)."""
    kx, kdx = axis_wavenumbers(n, L)
    ky, kdy = axis_wavenumbers(n, L)
    kz, kdz = axis_wavenumbers(n, L, half=True)
    kx, ky, kz = kx[:, None, None], ky[None, :, None], kz[None, None, :]
    kdx, kdy, kdz = kdx[:, None, None], kdy[None, :, None], kdz[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    return (kx, ky, kz), (kdx, kdy, kdz), k2


def fft3(a):
    return _sfft.rfftn(a, axes=(0, 1, 2), workers=FFT_WORKERS)


def ifft3(A, n):
    return _sfft.irfftn(A, s=(n, n, n), axes=(0, 1, 2), workers=FFT_WORKERS)


# --------------------------------------------------------------------------------------------
# Mass assignment (Sec. 3: binning of tracers on the mesh; CIC instead of the paper's NGP)
# --------------------------------------------------------------------------------------------
def _cic_corners(pos, n, L):
    """Yield (flat node index, weight) for the 8 CIC corners of every particle."""
    u = np.asarray(pos, dtype=np.float64) * (n / L)
    i0 = np.floor(u)
    t = u - i0
    i0 = i0.astype(np.int64)
    for dx in (0, 1):
        wx = t[:, 0] if dx else 1.0 - t[:, 0]
        ix = (i0[:, 0] + dx) % n
        for dy in (0, 1):
            wy = t[:, 1] if dy else 1.0 - t[:, 1]
            iy = (i0[:, 1] + dy) % n
            for dz in (0, 1):
                wz = t[:, 2] if dz else 1.0 - t[:, 2]
                iz = (i0[:, 2] + dz) % n
                yield (ix * n + iy) * n + iz, wx * wy * wz


def cic_deposit(pos, w, n: int, L: float):
    """rho on the n^3 nodes: sum over particles of w * prod_axis (1 - |u - i|)."""
    pos = np.asarray(pos, dtype=np.float64)
    w = np.ones(len(pos)) if w is None else np.asarray(w, dtype=np.float64)
    rho = np.zeros(n * n * n)
    for idx, cw in _cic_corners(pos, n, L):
        rho += np.bincount(idx, weights=w * cw, minlength=n ** 3)
    return rho.reshape(n, n, n)


def ngp_deposit(pos, w, n: int, L: float):
    """Nearest-grid-point binning (Sec. 3: the paper's scheme): each particle's weight goes to the
    node nearest to it, node i at x_i = i L / N, i.e. i = floor(x N / L + 1/2) modulo N."""
    pos = np.asarray(pos, dtype=np.float64)
    w = np.ones(len(pos)) if w is None else np.asarray(w, dtype=np.float64)
    i = np.floor(pos * (n / L) + 0.5).astype(np.int64) % n
    idx = (i[:, 0] * n + i[:, 1]) * n + i[:, 2]
    return np.bincount(idx, weights=w, minlength=n ** 3).reshape(n, n, n)


def radial_nbar(pos, observer, r_edges, sky_area: float):
    """Mean number density of a catalogue in radial shells about the observer (the n(z) of Sec. 3.2
    in comoving distance): counts per shell / (sky_area (r_hi^3 - r_lo^3) / 3), sky_area in sr."""
    r = np.sqrt(((np.asarray(pos, dtype=np.float64) - np.asarray(observer, dtype=np.float64)) ** 2).sum(1))
    counts, _ = np.histogram(r, bins=np.asarray(r_edges, dtype=np.float64))
    e = np.asarray(r_edges, dtype=np.float64)
    return counts / (sky_area * (e[1:] ** 3 - e[:-1] ** 3) / 3.0)


def fkp_weights(pos, observer, r_edges, nbar, P0: float = 20000.0):
    """FKP weights w = 1 / (1 + nbar(r) P0) (Sec. 3.2, P0 = 20000 (Mpc/h)^3), nbar of the shell that
    holds the particle's distance from the observer; particles outside the shells get nbar = 0."""
    r = np.sqrt(((np.asarray(pos, dtype=np.float64) - np.asarray(observer, dtype=np.float64)) ** 2).sum(1))
    e = np.asarray(r_edges, dtype=np.float64)
    b = np.searchsorted(e, r, side="right") - 1
    inside = (b >= 0) & (b < len(e) - 1)
    nb = np.zeros(len(r))
    nb[inside] = np.asarray(nbar, dtype=np.float64)[b[inside]]
    return 1.0 / (1.0 + nb * P0)


def cic_gather(field, pos, L: float):
    """Interpolate a real field (n,n,n) or (3,n,n,n) to particles with the CIC (trilinear) kernel."""
    field = np.asarray(field, dtype=np.float64)
    vec = field.ndim == 4
    n = field.shape[-1]
    flat = field.reshape(3, -1) if vec else field.reshape(1, -1)
    out = np.zeros((flat.shape[0], len(pos)))
    for idx, cw in _cic_corners(pos, n, L):
        out += flat[:, idx] * cw
    return out.T if vec else out[0]


# --------------------------------------------------------------------------------------------
# Overdensity, smoothing, mask, lognormal (Sec. 3.1, 3.2, 6)
# --------------------------------------------------------------------------------------------
def smooth(field, R: float, L: float):
    """Gaussian smoothing S(k) = exp(-k^2 R^2 / 2) applied in Fourier space (Sec. 3.1)."""
    n = field.shape[0]
    _, _, k2 = kgrid(n, L)
    return ifft3(fft3(field) * np.exp(-0.5 * k2 * R * R), n)


def overdensity_randoms(rho_g_s, rho_r_s, sum_wg: float, sum_wr: float, mask_frac: float,
                        n_touched: int):
    """delta = rho_g,s / (alpha rho_r,s) - 1 inside the survey mask, 0 outside (Sec. 3.2).

    alpha = sum w_g / sum w_r.  The binary mask keeps nodes where the smoothed random density exceeds
    mask_frac times the mean random density of the survey, sum w_r / n_touched, where n_touched is
    the number of nodes that received random mass in the (unsmoothed) deposit.
    Returns (delta, mask, alpha, threshold).
    """
    alpha = sum_wg / sum_wr
    thr = mask_frac * sum_wr / n_touched
    mask = rho_r_s > thr
    delta = np.zeros_like(rho_g_s)
    delta[mask] = rho_g_s[mask] / (alpha * rho_r_s[mask]) - 1.0
    return delta, mask, alpha, thr


def overdensity_uniform(rho_g_s, sum_wg: float):
    """delta = rho / rho_bar - 1 with rho_bar = sum w / N^3 (Sec. 2 definition, periodic box)."""
    rho_bar = sum_wg / rho_g_s.size
    return rho_g_s / rho_bar - 1.0


def lognormal(delta):
    """Eq. logdelta: delta -> ln(1 + delta) + C with C = -<ln(1 + delta)> (Sec. 6), 1+delta floored."""
    ld = np.log(np.maximum(1.0 + delta, LOG_FLOOR))
    return ld - ld.mean(), -ld.mean()


# --------------------------------------------------------------------------------------------
# Displacement operators (Eq. Zeldovich, Eq. Nusser)
# --------------------------------------------------------------------------------------------
def zeldovich_k(s_k, n: int, L: float):
    """Z[s] in Fourier space: the three components i kd_j s(k) / k^2, zero at k = 0."""
    _, kd, k2 = kgrid(n, L)
    inv = np.zeros_like(k2)
    np.divide(1.0, k2, out=inv, where=k2 > 0)
    return [1j * kd[j] * s_k * inv for j in range(3)]


def zeldovich(s, L: float):
    """Z[s] in configuration space: Psi with div Psi = -s (Eq. Zeldovich with s the source)."""
    n = s.shape[0]
    return np.stack([ifft3(c, n) for c in zeldovich_k(fft3(s), n, L)])


def divergence(v, L: float):
    """Spectral divergence of a real vector field v (3, n, n, n), returned in Fourier space."""
    n = v.shape[-1]
    _, kd, _ = kgrid(n, L)
    return sum(1j * kd[j] * fft3(v[j]) for j in range(3))


def rhat_field(n: int, L: float, observer, los_mode: int):
    """Unit line-of-sight vector at every node (Sec. 3.1: pointing away from the observer).

    Radial mode: (x_i - observer)/|x_i - observer|, zero at a node that coincides with the observer.
    Fixed mode: ``observer`` is read as the LOS direction and normalised (plane-parallel limit, Sec. 4.1).
    """
    o = np.asarray(observer, dtype=np.float64)
    if los_mode == LOS_FIXED:
        u = o / np.linalg.norm(o)
        return np.broadcast_to(u[:, None, None, None], (3, n, n, n)).copy()
    x = np.arange(n) * (L / n)
    d = np.stack(np.meshgrid(x - o[0], x - o[1], x - o[2], indexing="ij"))
    r = np.sqrt((d * d).sum(0))
    out = np.zeros_like(d)
    np.divide(d, r, out=out, where=r > 0)
    return out


def radial_projection(psi, rhat):
    """(Psi . r) r at every node."""
    u = (psi * rhat).sum(0)
    return u * rhat


def start_coefficient(start: int, beta: float) -> float:
    """Coefficient c of the starting estimate Psi_0 = Z[delta/b] - c (Z[delta/b].r) r.

    plain: 0; Eq. approx1: beta/(1+beta); Eq. approx2 (FFTA): 3 beta/(7 + 3 beta).  The paper writes
    f where this build uses beta = f/b.
    """
    if start == START_PLAIN:
        return 0.0
    if start == START_APPROX1:
        return beta / (1.0 + beta)
    if start == START_FFTA:
        return 3.0 * beta / (7.0 + 3.0 * beta)
    raise ValueError("unknown start")


def start_estimate(delta, b: float, f: float, L: float, rhat, start: int = START_PLAIN):
    """Starting estimate of Sec. 5.2: Psi_0 = Z[delta/b] - c (Z[delta/b].r) r, and Z[delta/b]."""
    psi_s = zeldovich(delta / b, L)
    c = start_coefficient(start, f / b)
    return psi_s - c * radial_projection(psi_s, rhat), psi_s


def update(psi, delta, b: float, f: float, L: float, rhat):
    """One step of Eq. iterative (Sec. 5.1): the estimate of the real-space delta/b,
    S = delta/b + beta div((Psi.r) r), and the new displacement Z[S] (Psi_FFT = -grad grad^-2 S)."""
    n = delta.shape[0]
    S_k = fft3(delta / b) + (f / b) * divergence(radial_projection(psi, rhat), L)
    return np.stack([ifft3(c_k, n) for c_k in zeldovich_k(S_k, n, L)])


def iterate(delta, b: float, f: float, L: float, rhat, start: int = START_PLAIN,
            tol: float = 0.0, max_iter: int = 6, return_all: bool = False):
    """Iterative solution of Eq. Nusser (Sec. 5.1, Eq. iterative), Psi in configuration space.

    Psi_0 is the starting estimate (plain or Eq. approx1/approx2).  For n = 0, 1, ...:
        S_n      = delta/b + beta div((Psi_n . r) r)        (estimate of the real-space delta / b)
        Psi_n+1  = Z[S_n]                                   (Psi_FFT,n+1 = -grad grad^-2 S_n)
    always restarting from the original delta.  rel[n] = |Psi_n+1 - Psi_n| / |Psi_n+1| (L2 over all
    nodes and components), except rel[0], which is measured against the uncorrected estimate
    Z[delta/b] for every start.  Stops when rel[n] < tol with n >= 1, or after max_iter updates.
    Returns (Psi_final (3,n,n,n), rel list, n_updates[, list of all Psi_n]).
    """
    psi, prev_for_rel = start_estimate(delta, b, f, L, rhat, start)
    rels, history = [], [psi]
    it = 0
    while it < max_iter:
        psi_new = update(psi, delta, b, f, L, rhat)
        num = np.sqrt(((psi_new - prev_for_rel) ** 2).sum())
        den = np.sqrt((psi_new ** 2).sum())
        rels.append(num / den if den > 0 else 0.0)
        psi = psi_new
        prev_for_rel = psi_new
        history.append(psi)
        it += 1
        if it >= 2 and rels[-1] < tol:
            break
    if return_all:
        return psi, rels, it, history
    return psi, rels, it


# --------------------------------------------------------------------------------------------
# Reconstruction shift (Sec. 1: move galaxies and randoms back along the displacement)
# --------------------------------------------------------------------------------------------
def particle_rhat(pos, observer, los_mode: int):
    o = np.asarray(observer, dtype=np.float64)
    if los_mode == LOS_FIXED:
        u = o / np.linalg.norm(o)
        return np.broadcast_to(u, np.shape(pos)).copy()
    d = np.asarray(pos, dtype=np.float64) - o
    r = np.sqrt((d * d).sum(1))[:, None]
    out = np.zeros_like(d)
    np.divide(d, r, out=out, where=r > 0)
    return out


def shift_vectors(psi, pos, L: float, f: float, observer, los_mode: int, is_galaxy: bool, periodic: bool = False):
    """Shift d = -[Psi + f (Psi.r) r] for galaxies and d = -Psi for randoms, Psi CIC-interpolated.

    In a periodic box a position stands for its image in [0, L): the line of sight runs from the
    observer to that image (the interpolation is periodic either way)."""
    p = cic_gather(psi, pos, L)
    if not is_galaxy:
        return -p
    rh = particle_rhat(np.mod(pos, L) if periodic else pos, observer, los_mode)
    u = (p * rh).sum(1)[:, None]
    return -(p + f * u * rh)


def shifted_positions(pos, d, L: float, periodic: bool):
    x = np.asarray(pos, dtype=np.float64) + d
    return np.mod(x, L) if periodic else x


# --------------------------------------------------------------------------------------------
# Finite-difference configuration-space method (Sec. 2.1, Eq. mainpot)
# --------------------------------------------------------------------------------------------
def _shift(a, d):
    """a at the node offset by d = (dx, dy, dz), zero beyond the mesh: out[i] = a[i + d] (the
    finite-difference problem's boundary condition phi = 0 outside the box)."""
    out = np.zeros_like(a)
    src = tuple(slice(max(0, k), a.shape[j] + min(0, k)) for j, k in enumerate(d))
    dst = tuple(slice(max(0, -k), a.shape[j] + min(0, -k)) for j, k in enumerate(d))
    out[dst] = a[src]
    return out


def fd_operator(phi, L: float, beta: float, observer, los_mode: int):
    """A phi = grad^2 phi + beta div((grad phi . r) r) on the mesh, phi = 0 outside it, with the
    stencils of Sec. 2.1: the 7-point Laplacian (set A) and, for the line-of-sight term,
      -2 phi_0 / g^2 + sum_B (x_i^2 / (g^2 r^2) +- x_i / (g r^2)) phi_(+-i)
                     + sum_C (-1)^p x_i x_j / (2 g^2 r^2) phi_(+-i, +-j)
    with x the node's offset from the observer, r = |x|, g the mesh spacing, p = 0 when the two
    offsets have the same sign and 1 otherwise (the paper writes f where this build uses beta).  For
    a fixed line of sight u the term is sum_ij u_i u_j d_i d_j phi with the same second-difference
    stencils (x_i / r -> u_i, no 1/r term).  At the observer's node the term is 0."""
    n = phi.shape[0]
    g = L / n
    out = -6.0 * phi
    for a in range(3):
        for sgn in (1, -1):
            d = [0, 0, 0]
            d[a] = sgn
            out = out + _shift(phi, d)
    out = out / (g * g)
    if beta == 0.0:
        return out
    if los_mode == LOS_FIXED:
        u = np.asarray(observer, dtype=np.float64)
        u = u / np.linalg.norm(u)
        xs = [np.full(phi.shape, u[a]) for a in range(3)]
        inv_r2 = np.ones(phi.shape)
        first = 0.0
    else:
        o = np.asarray(observer, dtype=np.float64)
        x = np.arange(n) * g
        xs = list(np.meshgrid(x - o[0], x - o[1], x - o[2], indexing="ij"))
        r2 = xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2
        inv_r2 = np.zeros_like(r2)
        np.divide(1.0, r2, out=inv_r2, where=r2 > 0)
        first = 1.0
    rsd = -2.0 * phi * (inv_r2 > 0) / (g * g)
    for a in range(3):
        for sgn in (1, -1):
            d = [0, 0, 0]
            d[a] = sgn
            coef = xs[a] ** 2 * inv_r2 / (g * g) + sgn * first * xs[a] * inv_r2 / g
            rsd = rsd + coef * _shift(phi, d)
    for a in range(3):
        for b in range(a + 1, 3):
            for sa in (1, -1):
                for sb in (1, -1):
                    d = [0, 0, 0]
                    d[a], d[b] = sa, sb
                    rsd = rsd + (sa * sb) * xs[a] * xs[b] * inv_r2 / (2.0 * g * g) * _shift(phi, d)
    return out + beta * rsd


def fd_laplacian_eigen(n: int, L: float):
    """Eigenvalues of the periodic 7-point Laplacian on the rfftn grid: sum_i (2 cos(k_i g) - 2) / g^2."""
    g = L / n
    (kx, ky, kz), _, _ = kgrid(n, L)
    return sum((2.0 * np.cos(k * g) - 2.0) / (g * g) for k in (kx, ky, kz))


def fd_solve(delta, b: float, f: float, L: float, observer, los_mode: int, tol: float = 1e-10,
             max_iter: int = 500):
    """The configuration-space method of Sec. 2.1: solve A phi = delta/b (A as fd_operator, the
    paper's A phi = delta_g / b with Psi = -grad phi, phi = 0 outside the box) with GMRES,
    preconditioned by the inverse of the periodic 7-point Laplacian (applied with FFTs); then
    Psi = -grad phi by central differences (phi = 0 beyond the box).  Returns (Psi, phi,
    iterations, relative residual)."""
    from scipy.sparse.linalg import LinearOperator, gmres
    n = delta.shape[0]
    beta = f / b
    rhs = delta / b
    lam = fd_laplacian_eigen(n, L)
    inv_lam = np.zeros_like(lam)
    np.divide(1.0, lam, out=inv_lam, where=lam != 0)
    inv_lam[0, 0, 0] = -L * L / (3.0 * np.pi ** 2)   # the constant mode: the lowest Dirichlet eigenvalue
    shape = delta.shape
    A = LinearOperator((n ** 3, n ** 3), dtype=np.float64,
                       matvec=lambda v: fd_operator(v.reshape(shape), L, beta, observer, los_mode).ravel())
    M = LinearOperator((n ** 3, n ** 3), dtype=np.float64,
                       matvec=lambda v: ifft3(fft3(v.reshape(shape)) * inv_lam, n).ravel())
    count = [0]

    def cb(_):
        count[0] += 1
    sol, info = gmres(A, rhs.ravel(), M=M, rtol=tol, atol=0.0, restart=50, maxiter=max_iter,
                      callback=cb, callback_type="pr_norm")
    phi = sol.reshape(shape)
    res = np.linalg.norm(fd_operator(phi, L, beta, observer, los_mode) - rhs) / np.linalg.norm(rhs)
    g = L / n
    psi = np.stack([-(_shift(phi, [1 if a == j else 0 for a in range(3)]) -
                      _shift(phi, [-1 if a == j else 0 for a in range(3)])) / (2.0 * g) for j in range(3)])
    return psi, phi, count[0], res


# --------------------------------------------------------------------------------------------
# Diagnostics of the paper (Sec. 4.1 Helmholtz split, Sec. 4.3 / 5.2 radial ratio)
# --------------------------------------------------------------------------------------------
RATIO_LO, RATIO_HI = -1.0, 3.0   # Tables 1-3: ratios above 3 or below -1 are outliers


def converged_at(means, tol: float = 0.01):
    """The convergence rule of Sec. 5.2 (captions of Tables 2 and 3) on a sequence of mean ratios
    m_0, m_1, ...: the first iteration n after which every mean differs from the one before it by
    at most tol, |m_(k+1) - m_k| <= tol for all k >= n (the last iteration qualifies when no earlier
    one does).  Reading: the ratios are near 1, so the paper's 1% is taken as an absolute 0.01, and
    "at most" rather than "less than" because only then do the paper's printed two-decimal tables
    give the iteration counts it states (Table 2: 4 and 2, Table 3: 6 and 2)."""
    m = [float(x) for x in means]
    for n in range(len(m)):
        if all(abs(m[k + 1] - m[k]) <= tol + 1e-12 for k in range(n, len(m) - 1)):
            return n
    return len(m) - 1


def ratio_stats(num, den, lo: float = RATIO_LO, hi: float = RATIO_HI):
    """Mean and standard deviation of the ratio num/den over all points, outliers removed (Table 1-3
    rule: a ratio above hi or below lo; a zero denominator counts as an outlier).  Returns
    (mean, std, outlier fraction, number kept); std is the population value of the kept ratios."""
    num = np.asarray(num, dtype=np.float64).ravel()
    den = np.asarray(den, dtype=np.float64).ravel()
    ok = den != 0
    r = num[ok] / den[ok]
    keep = (r >= lo) & (r <= hi)
    kept = r[keep]
    n_keep = kept.size
    mean = kept.mean() if n_keep else 0.0
    std = kept.std() if n_keep else 0.0
    return mean, std, 1.0 - n_keep / num.size, n_keep


def radial_ratio(psi_real, psi_est, pos, L: float, observer, los_mode: int, periodic: bool = False,
                 lo: float = RATIO_LO, hi: float = RATIO_HI):
    """Eq. ratio at particle positions: (Psi_real . r) / (Psi_est . r), both fields CIC-interpolated
    to each particle and projected on the particle's line of sight; statistics as ratio_stats."""
    rh = particle_rhat(np.mod(pos, L) if periodic else pos, observer, los_mode)
    a = (cic_gather(psi_real, pos, L) * rh).sum(1)
    b = (cic_gather(psi_est, pos, L) * rh).sum(1)
    return ratio_stats(a, b, lo, hi)


def helmholtz_x(psi, L: float):
    """Sec. 4.1, plane-parallel split of (Psi.x) x with Psi_x = Psi.x (Eq. Helmholtz): in Fourier
    space the irrotational part grad A has components (k_j k_x / k^2) Psi_x(k) (Eq. irrotational)
    and the solenoidal part curl B = (Psi.x) x - grad A (Eq. solenoidal: ((k_y^2 + k_z^2) / k^2,
    -k_y k_x / k^2, -k_z k_x / k^2) Psi_x(k)).  Derivative wavenumbers as in the rest of the oracle
    (zero at the Nyquist index); k = 0 carries no irrotational part.  Returns (grad_A, curl_B),
    each (3, n, n, n)."""
    n = psi.shape[-1]
    _, kd, k2 = kgrid(n, L)
    inv = np.zeros_like(k2)
    np.divide(1.0, k2, out=inv, where=k2 > 0)
    Px = fft3(psi[0])
    grad_a = np.stack([ifft3(kd[j] * kd[0] * inv * Px, n) for j in range(3)])
    curl_b = -grad_a
    curl_b[0] += psi[0]
    return grad_a, curl_b


# --------------------------------------------------------------------------------------------
# Whole pipeline (what recon_deposit -> smooth -> iterate -> shift computes)
# --------------------------------------------------------------------------------------------
def reconstruct(params: dict, gal_pos, gal_w=None, ran_pos=None, ran_w=None,
                start: int = START_PLAIN, tol: float = 0.0, max_iter: int = 6,
                shift: bool = True, mask_flip=None):
    """Run the whole method on a catalogue; returns a dict of every intermediate.

    params: n, L, b, f, R, los_mode, observer, periodic, mask_frac, lognormal, uniform (bool), and
    optionally ngp (bool: the paper's nearest-grid-point binning instead of CIC, Sec. 3).
    mask_flip: optional flat node indices at which the survey-mask decision is inverted.  The mask
    is a floating-point comparison of the smoothed random density with a threshold; at nodes whose
    density lies within rounding of the threshold either decision is valid, and a comparison with
    a float32 implementation picks the branch that implementation took there.
    """
    n, L = int(params["n"]), float(params["L"])
    gal_pos = np.asarray(gal_pos, dtype=np.float64)
    wg = np.ones(len(gal_pos)) if gal_w is None else np.asarray(gal_w, dtype=np.float64)
    out = {}
    deposit = ngp_deposit if params.get("ngp", False) else cic_deposit
    rho_g = deposit(gal_pos, wg, n, L)
    out["rho_g"] = rho_g
    out["sum_wg"] = wg.sum()
    rho_g_s = smooth(rho_g, params["R"], L)
    if params.get("uniform", False):
        delta = overdensity_uniform(rho_g_s, wg.sum())
        out["mask"] = np.ones(delta.shape, dtype=bool)
    else:
        ran_pos = np.asarray(ran_pos, dtype=np.float64)
        wr = np.ones(len(ran_pos)) if ran_w is None else np.asarray(ran_w, dtype=np.float64)
        rho_r = deposit(ran_pos, wr, n, L)
        out["rho_r"] = rho_r
        out["sum_wr"] = wr.sum()
        rho_r_s = smooth(rho_r, params["R"], L)
        out["rho_r_s"] = rho_r_s
        delta, mask, alpha, thr = overdensity_randoms(rho_g_s, rho_r_s, wg.sum(), wr.sum(),
                                                      params.get("mask_frac", 0.01),
                                                      int(np.count_nonzero(rho_r > 0)))
        if mask_flip is not None and len(mask_flip):
            mask = mask.copy()
            mf = mask.reshape(-1)
            idx = np.asarray(mask_flip, dtype=np.int64)
            mf[idx] = ~mf[idx]
            delta = np.zeros_like(rho_g_s)
            delta[mask] = rho_g_s[mask] / (alpha * rho_r_s[mask]) - 1.0
        out.update(mask=mask, alpha=alpha, threshold=thr)
    out["rho_g_s"] = rho_g_s
    if params.get("lognormal", False):
        delta, C = lognormal(delta)
        out["lognormal_C"] = C
    out["delta"] = delta
    rhat = rhat_field(n, L, params["observer"], params.get("los_mode", LOS_RADIAL))
    psi, rels, it = iterate(delta, params["b"], params["f"], L, rhat, start, tol, max_iter)
    out.update(psi=psi, rel=rels, n_iter=it)
    if shift:
        periodic = bool(params.get("periodic", False))
        dg = shift_vectors(psi, gal_pos, L, params["f"], params["observer"],
                           params.get("los_mode", LOS_RADIAL), True, periodic)
        out["shift_g"] = dg
        out["pos_g"] = shifted_positions(gal_pos, dg, L, periodic)
        if ran_pos is not None:
            dr = shift_vectors(psi, ran_pos, L, params["f"], params["observer"],
                               params.get("los_mode", LOS_RADIAL), False)
            out["shift_r"] = dr
            out["pos_r"] = shifted_positions(ran_pos, dr, L, periodic)
    return out
