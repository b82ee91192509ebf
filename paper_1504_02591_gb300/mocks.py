"""Seeded synthetic catalogues shaped like the workloads of Burden, Percival & Howlett (2015).

The paper's own inputs (a GADGET-2 N-body run, Sec. 3.1; PTHalo BOSS DR11 CMASS mocks, Sec. 3.2) are
not available, so these generators stand in for them with the same shapes: box, mesh, tracer counts,
random-to-galaxy ratio, survey-like shell windows and a radial line of sight.

Recipe: a Gaussian random field with P(k) = A k^-1.5 exp(-(k/0.3)^2) (A chosen so that the field
smoothed with a Gaussian of R = 15 Mpc/h has unit variance) is drawn on a coarse generator grid from
seeded normal noise.  Its first-order displacement moves Lagrangian points q (a jittered lattice or
uniform points) to x = q + D(q); galaxies are kept with probability proportional to
max(0, 1 + (b - 1) delta_L(q)) (Lagrangian bias) and moved to redshift space by s = x + f (D.r) r.
Randoms are uniform in the same window.  Optionally (k_turn) the spectrum is turned over to P ~ k
below k_turn, which bounds the bulk flows that the k^-1.5 spectrum drives from scales larger than a
survey window.

This module is input plumbing only.  It is shared by the tests, the benchmark and the oracle runs, and
it contains no code of either the CUDA path or the oracle; its small Fourier-space displacement and
trilinear interpolation are its own.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

try:  # threaded FFTs when scipy is present; numpy otherwise (same results up to rounding)
    import scipy.fft as _sfft

    def _rfftn(a):
        return _sfft.rfftn(a, workers=-1)

    def _irfftn(a, s):
        return _sfft.irfftn(a, s=s, workers=-1)
except Exception:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)

PK_AMPLITUDE = 1940.5   # (Mpc/h)^1.5: sigma(R = 15 Mpc/h) = 1 for the spectrum below
PK_SLOPE = -1.5
PK_CUTOFF = 0.3         # h/Mpc


def power_spectrum(k, k_turn: float | None = None):
    """A k^-1.5 exp(-(k/0.3)^2); with k_turn, times x/(1 + x), x = (k/k_turn)^2.5, which turns the
    spectrum over to P ~ k at k << k_turn (as a CDM spectrum does near its peak) and so bounds the
    large-scale (bulk-flow) part of the displacement."""
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros_like(k)
    pos = k > 0
    out[pos] = PK_AMPLITUDE * k[pos] ** PK_SLOPE * np.exp(-(k[pos] / PK_CUTOFF) ** 2)
    if k_turn:
        x = (k[pos] / k_turn) ** 2.5
        out[pos] *= x / (1.0 + x)
    return out


@dataclass
class GeneratorField:
    """Linear density and displacement on a periodic generator grid."""
    ng: int
    L: float
    delta: np.ndarray            # (ng, ng, ng) float32
    disp: np.ndarray             # (3, ng, ng, ng) float32

    def sample(self, pts):
        """Trilinear interpolation of (delta, disp) at points (n, 3); periodic."""
        u = np.asarray(pts, dtype=np.float64) * (self.ng / self.L)
        f0 = np.floor(u)
        t = (u - f0).astype(np.float32)
        i0 = f0.astype(np.int64) % self.ng
        i1 = (i0 + 1) % self.ng
        d = np.zeros(len(u), dtype=np.float32)
        v = np.zeros((len(u), 3), dtype=np.float32)
        for cx in (0, 1):
            ix = i1[:, 0] if cx else i0[:, 0]
            wx = t[:, 0] if cx else 1 - t[:, 0]
            for cy in (0, 1):
                iy = i1[:, 1] if cy else i0[:, 1]
                wy = t[:, 1] if cy else 1 - t[:, 1]
                for cz in (0, 1):
                    iz = i1[:, 2] if cz else i0[:, 2]
                    wz = t[:, 2] if cz else 1 - t[:, 2]
                    w = wx * wy * wz
                    d += w * self.delta[ix, iy, iz]
                    for a in range(3):
                        v[:, a] += w * self.disp[a, ix, iy, iz]
        return d, v


def gaussian_field(ng: int, L: float, seed: int, amp: float = 1.0, k_turn: float | None = None) -> GeneratorField:
    """The field of the spectrum above times amp (amp < 1: closer to the linear regime), turned over
    below k_turn when given."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((ng, ng, ng), dtype=np.float32)
    W = _rfftn(white)
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    mz = np.arange(ng // 2 + 1)
    kf = 2 * np.pi / L
    kx = (kf * m)[:, None, None]
    ky = (kf * m)[None, :, None]
    kz = (kf * mz)[None, None, :]
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    vcell = (L / ng) ** 3
    D = W * (amp * np.sqrt(power_spectrum(kk, k_turn) / vcell))
    D[0, 0, 0] = 0
    delta = _irfftn(D, (ng, ng, ng)).astype(np.float32)
    inv_k2 = np.zeros_like(kk)
    np.divide(1.0, kk ** 2, out=inv_k2, where=kk > 0)
    disp = np.empty((3, ng, ng, ng), dtype=np.float32)
    for a, ka in enumerate((kx, ky, kz)):
        disp[a] = _irfftn(1j * ka * D * inv_k2, (ng, ng, ng))
    return GeneratorField(ng, L, delta, disp)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    r = np.sqrt((v * v).sum(-1, keepdims=True))
    return np.divide(v, r, out=np.zeros_like(v), where=r > 0)


@dataclass
class Catalog:
    pos: np.ndarray                      # (n, 3) float64, Mpc/h
    w: np.ndarray | None = None          # (n,) float32 or None (unit weights)


@dataclass
class Mock:
    name: str
    L: float
    n_mesh: int
    b: float
    f: float
    R: float
    observer: tuple
    los_mode: int = 0                    # 0 radial, 1 fixed (observer read as a direction)
    periodic: bool = True
    uniform: bool = False                # mean density from N^3 instead of randoms
    galaxies: Catalog | None = None
    randoms: Catalog | None = None
    window: dict = field(default_factory=dict)
    galaxies_real: Catalog | None = None  # the same galaxies before the redshift-space shift

    def params(self, **over):
        p = dict(n=self.n_mesh, L=self.L, b=self.b, f=self.f, R=self.R, observer=self.observer,
                 los_mode=self.los_mode, periodic=self.periodic, uniform=self.uniform,
                 mask_frac=0.01, lognormal=False)
        p.update(over)
        return p


def _rsd(x, v, f, observer, los_mode):
    if los_mode == 1:
        rh = np.broadcast_to(_unit(np.asarray(observer, dtype=np.float64)), x.shape)
    else:
        rh = _unit(x - np.asarray(observer, dtype=np.float64))
    return x + f * (v * rh).sum(1, keepdims=True) * rh


def periodic_box(L: float, n_mesh: int, n_gal: int, n_ran: int, b: float, f: float, R: float,
                 observer, seed_field: int, seed_gal: int, seed_ran: int, ng: int | None = None,
                 los_mode: int = 0, uniform: bool = False, name: str = "periodic") -> Mock:
    """Periodic box: galaxies from a jittered lattice, Zel'dovich-displaced, biased, RSD-shifted."""
    ng = ng or min(n_mesh, 256)
    gf = gaussian_field(ng, L, seed_field)
    rng = np.random.default_rng(seed_gal)
    # lattice with enough sites that the biased selection can keep n_gal of them
    side = int(np.ceil((2.0 * n_gal) ** (1.0 / 3.0)))
    g = (np.arange(side) + 0.5) * (L / side)
    q = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    q = q + rng.uniform(-0.5, 0.5, q.shape) * (L / side)          # jitter inside the lattice cell
    dl, v = gf.sample(q)
    p_keep = np.maximum(0.0, 1.0 + (b - 1.0) * dl.astype(np.float64))
    p_keep /= p_keep.max()
    # keep the n_gal sites with the smallest u/p (a weighted draw without replacement)
    key = rng.uniform(size=len(q)) / np.maximum(p_keep, 1e-12)
    sel = np.argsort(key)[:n_gal]
    x = q[sel] + v[sel].astype(np.float64)
    s = np.mod(_rsd(x, v[sel].astype(np.float64), f, observer, los_mode), L)
    mock = Mock(name, L, n_mesh, b, f, R, tuple(observer), los_mode, True, uniform,
                galaxies=Catalog(s), galaxies_real=Catalog(np.mod(x, L)))
    if n_ran > 0:
        rr = np.random.default_rng(seed_ran)
        mock.randoms = Catalog(rr.uniform(0.0, L, (n_ran, 3)))
    return mock


def _in_window(p, observer, axis, r_min, r_max, cos_min):
    d = p - np.asarray(observer)
    r = np.sqrt((d * d).sum(1))
    c = (d @ np.asarray(axis)) / np.maximum(r, 1e-30)
    return (r >= r_min) & (r <= r_max) & (c >= cos_min)


def shell_survey(L: float, n_mesh: int, n_gal: int, n_ran: int, b: float, f: float, R: float,
                 observer, axis, r_min: float, r_max: float, sky_frac: float,
                 seed_field: int, seed_gal: int, seed_ran: int, ng: int | None = None,
                 name: str = "shell", amp: float = 1.0, k_turn: float | None = None) -> Mock:
    """Spherical-shell cap window (r_min..r_max around the observer, sky fraction sky_frac)."""
    ng = ng or min(n_mesh, 256)
    gf = gaussian_field(ng, L, seed_field, amp, k_turn)
    obs = np.asarray(observer, dtype=np.float64)
    ax = _unit(np.asarray(axis, dtype=np.float64))
    cos_min = 1.0 - 2.0 * sky_frac
    # bounding box of the window, widened by a displacement margin
    margin = 80.0
    lo = np.clip(obs - r_max - margin, 0, L)
    hi = np.clip(obs + r_max + margin, 0, L)
    sin_max = np.sqrt(max(0.0, 1 - cos_min ** 2))
    for a in range(3):  # tighten along the cap axis when it is a coordinate axis
        if abs(ax[a]) > 0.999:
            if ax[a] > 0:
                lo[a] = max(lo[a], obs[a] + r_min * cos_min - margin)
            else:
                hi[a] = min(hi[a], obs[a] - r_min * cos_min + margin)
    del sin_max
    rng = np.random.default_rng(seed_gal)
    got, chunks, real = 0, [], []
    vol_box = np.prod(hi - lo)
    vol_win = sky_frac * 4.0 / 3.0 * np.pi * (r_max ** 3 - r_min ** 3)
    per = int(n_gal * 2.0 * vol_box / vol_win) + 1000
    while got < n_gal:
        q = lo + rng.uniform(size=(per, 3)) * (hi - lo)
        dl, v = gf.sample(q)
        p_keep = np.maximum(0.0, 1.0 + (b - 1.0) * dl.astype(np.float64))
        keep = rng.uniform(size=per) * 4.0 < p_keep          # thinning; 4 bounds 1+(b-1)delta
        q, v = q[keep], v[keep].astype(np.float64)
        s = _rsd(q + v, v, f, obs, 0)
        inw = _in_window(s, obs, ax, r_min, r_max, cos_min)
        chunks.append(s[inw])
        real.append((q + v)[inw])
        got += int(inw.sum())
    gal = np.concatenate(chunks)[:n_gal]
    rr = np.random.default_rng(seed_ran)
    u = rr.uniform(size=(n_ran, 3))
    r = np.cbrt(u[:, 0] * (r_max ** 3 - r_min ** 3) + r_min ** 3)
    ct = cos_min + u[:, 1] * (1.0 - cos_min)
    st = np.sqrt(np.maximum(0.0, 1 - ct * ct))
    ph = 2 * np.pi * u[:, 2]
    # orthonormal frame around the cap axis
    t1 = _unit(np.cross(ax, [0.0, 0.0, 1.0]) if abs(ax[2]) < 0.9 else np.cross(ax, [1.0, 0.0, 0.0]))
    t2 = np.cross(ax, t1)
    dirs = ct[:, None] * ax + (st * np.cos(ph))[:, None] * t1 + (st * np.sin(ph))[:, None] * t2
    ran = obs + r[:, None] * dirs
    mock = Mock(name, L, n_mesh, b, f, R, tuple(obs), 0, False, False,
                galaxies=Catalog(gal), randoms=Catalog(ran),
                window=dict(axis=tuple(ax), r_min=r_min, r_max=r_max, sky_frac=sky_frac),
                galaxies_real=Catalog(np.concatenate(real)[:n_gal]))
    return mock


# ---------------------------------------------------------------------------------------------
# The workloads (sizes and parameters as the paper's data sets and the build's configurations)
# ---------------------------------------------------------------------------------------------
def small_periodic(n_gal: int = 200_000, n_ran: int = 2_000_000, n_mesh: int = 64) -> Mock:
    """64^3 periodic box, L = 1000 Mpc/h, 2e5 galaxies, 2e6 randoms, b = 2, f = 0.74, R = 15,
    observer at the box centre offset by 1500 Mpc/h along x."""
    return periodic_box(1000.0, n_mesh, n_gal, n_ran, 2.0, 0.74, 15.0, (2000.0, 500.0, 500.0),
                        1, 2, 3, ng=128, name="periodic-64")


def survey_shell_512(n_gal: int = 600_000, ran_ratio: int = 50, n_mesh: int = 512,
                     L: float = 3500.0, seed: int = 10, amp: float = 1.0,
                     k_turn: float | None = None) -> Mock:
    """512^3 mesh in a 3500 Mpc/h box, shell 1100-1800 Mpc/h, 25% sky cap, 6e5 galaxies, 50x
    randoms, b = 1.85, f = 0.74, R = 15.  Observer at the centre of the x = 0 face, cap axis +x
    (a box-corner observer sees at most 1/8 of the sky, so a 25% cap cannot sit at the corner).
    Seeds seed, seed + 1, seed + 2 (field, galaxies, randoms); the benchmark mock is seed 10.
    amp scales the field; k_turn turns the spectrum over at large scales (the diagnostics' mocks)."""
    return shell_survey(L, n_mesh, n_gal, n_gal * ran_ratio, 1.85, 0.74, 15.0,
                        (0.0, L / 2, L / 2), (1.0, 0.0, 0.0), 1100.0, 1800.0, 0.25,
                        seed, seed + 1, seed + 2, ng=256, name=f"shell-{n_mesh}", amp=amp, k_turn=k_turn)


def scaled_shell(n_mesh: int, L: float, n_gal: int, ran_ratio: int, b: float, f: float,
                 seed: int) -> Mock:
    """Shell survey scaled to box L (distances scaled from the 3500 Mpc/h shape)."""
    s = L / 3500.0
    return shell_survey(L, n_mesh, n_gal, n_gal * ran_ratio, b, f, 15.0, (0.0, L / 2, L / 2),
                        (1.0, 0.0, 0.0), 1100.0 * s, 1800.0 * s, 0.25, seed, seed + 1, seed + 2,
                        ng=min(256, n_mesh), name=f"shell-{n_mesh}-{seed}")


def lattice_box(L: float, n_mesh: int, side: int, n_total: int, b: float, f: float, R: float,
                observer, los_mode: int, seed: int, device: str = "cuda", name: str = "lattice") -> Mock:
    """Periodic box of Zel'dovich-displaced particles, generated with torch on `device`.

    A Gaussian field with the spectrum above is drawn on the side^3 lattice itself (nodes
    q = i L / side), so each node is displaced by the field's first-order displacement D(q) without
    interpolation; the n_total - side^3 further particles are randomly chosen nodes jittered
    uniformly within half a lattice cell, displaced like their node.  Redshift-space positions
    s = x + f (D.r) r are wrapped into [0, L).  Uniform mean density (no randoms); with b = 1 every
    particle is kept.  Returns float64 positions on the host."""
    import torch
    gen = torch.Generator(device=device).manual_seed(seed)
    white = torch.randn((side, side, side), generator=gen, device=device, dtype=torch.float32)
    W = torch.fft.rfftn(white)
    del white
    kf = 2 * np.pi / L
    m = torch.fft.fftfreq(side, d=1.0 / side, device=device, dtype=torch.float64)
    mz = torch.arange(side // 2 + 1, device=device, dtype=torch.float64)
    kx, ky, kz = (kf * m)[:, None, None], (kf * m)[None, :, None], (kf * mz)[None, None, :]
    kk = torch.sqrt(kx * kx + ky * ky + kz * kz)
    pos_k = kk > 0
    pk = torch.where(pos_k, PK_AMPLITUDE * torch.where(pos_k, kk, 1.0) ** PK_SLOPE
                     * torch.exp(-(kk / PK_CUTOFF) ** 2), torch.zeros_like(kk))
    amp = torch.sqrt(pk / (L / side) ** 3) / torch.where(pos_k, kk * kk, 1.0)
    amp[0, 0, 0] = 0.0
    D = W * amp.to(torch.float32)
    del W, pk, amp
    disp = torch.empty((side ** 3, 3), device=device, dtype=torch.float64)
    for a, ka in enumerate((kx, ky, kz)):
        disp[:, a] = torch.fft.irfftn(1j * ka.to(torch.float32) * D, s=(side,) * 3).reshape(-1).double()
    del D
    g = torch.arange(side, device=device, dtype=torch.float64) * (L / side)
    q = torch.stack(torch.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    extra = max(0, n_total - side ** 3)
    if extra:
        pick = torch.randint(0, side ** 3, (extra,), generator=gen, device=device)
        jit = (torch.rand((extra, 3), generator=gen, device=device, dtype=torch.float64) - 0.5) * (L / side)
        q = torch.cat([q, q[pick] + jit])
        disp = torch.cat([disp, disp[pick]])
    x = q + disp
    del q
    obs = torch.tensor(observer, device=device, dtype=torch.float64)
    if los_mode == 1:
        rh = (obs / torch.linalg.norm(obs)).expand_as(x)
    else:
        d = x - obs
        rh = d / torch.linalg.norm(d, dim=1, keepdim=True).clamp_min(1e-30)
        del d
    s = torch.remainder(x + f * (disp * rh).sum(1, keepdim=True) * rh, L)
    del x, disp, rh
    pos = s[:n_total].cpu().numpy()
    return Mock(name, L, n_mesh, b, f, R, tuple(observer), los_mode, True, True, galaxies=Catalog(pos))


def large_periodic_1024(los_mode: int = 0, n_mesh: int = 1024, side: int = 464,
                        n_total: int = 100_000_000, device: str = "cuda") -> Mock:
    """The large periodic run: 2500 Mpc/h box, 1024^3 mesh, 1e8 particles (a 464^3 lattice plus
    102,656 jittered copies of lattice nodes), b = 1, f = 0.74, R = 10, uniform mean density.
    Radial line of sight from (-1000, 1250, 1250), or (los_mode = 1) the fixed direction +x."""
    obs = (1.0, 0.0, 0.0) if los_mode == 1 else (-1000.0, 1250.0, 1250.0)
    return lattice_box(2500.0, n_mesh, side, n_total, 1.0, 0.74, 10.0, obs, los_mode, 20, device=device,
                       name=f"periodic-{n_mesh}-{'fixed' if los_mode else 'radial'}")


# ---------------------------------------------------------------------------------------------
# Batches of mocks generated on the GPU (the batched workload: dozens of catalogues of up to 5e7
# tracers each, too many to draw with numpy in a benchmark's time).  Same recipe as above, with
# torch's seeded generators: Gaussian field on a generator grid, trilinear displacement and
# overdensity at uniform Lagrangian points, biased thinning, redshift-space shift along the radial
# line of sight, shell-cap window or periodic wrap; randoms uniform in the window.
# ---------------------------------------------------------------------------------------------
def _field_device(ng, L, gen, device):
    import torch
    white = torch.randn((ng, ng, ng), generator=gen, device=device, dtype=torch.float32)
    W = torch.fft.rfftn(white)
    kf = 2 * np.pi / L
    m = torch.fft.fftfreq(ng, d=1.0 / ng, device=device, dtype=torch.float64)
    mz = torch.arange(ng // 2 + 1, device=device, dtype=torch.float64)
    kx, ky, kz = (kf * m)[:, None, None], (kf * m)[None, :, None], (kf * mz)[None, None, :]
    kk = torch.sqrt(kx * kx + ky * ky + kz * kz)
    pos_k = kk > 0
    ksafe = torch.where(pos_k, kk, torch.ones_like(kk))
    pk = torch.where(pos_k, PK_AMPLITUDE * ksafe ** PK_SLOPE * torch.exp(-(kk / PK_CUTOFF) ** 2), torch.zeros_like(kk))
    D = W * torch.sqrt(pk / (L / ng) ** 3).to(torch.float32)
    fields = [torch.fft.irfftn(D, s=(ng,) * 3)]
    inv_k2 = torch.where(pos_k, 1.0 / (ksafe * ksafe), torch.zeros_like(kk)).to(torch.float32)
    for ka in (kx, ky, kz):
        fields.append(torch.fft.irfftn(1j * ka.to(torch.float32) * D * inv_k2, s=(ng,) * 3))
    return torch.stack(fields)                 # (4, ng, ng, ng): delta, D_x, D_y, D_z


def _trilinear_device(F, pts, L):
    """F (c, ng, ng, ng) at points (n, 3), periodic; returns (n, c)."""
    import torch
    ng = F.shape[-1]
    u = pts * (ng / L)
    f0 = torch.floor(u)
    t = (u - f0).to(torch.float32)
    i0 = f0.long() % ng
    i1 = (i0 + 1) % ng
    flat = F.reshape(F.shape[0], -1)
    out = torch.zeros((pts.shape[0], F.shape[0]), device=pts.device, dtype=torch.float32)
    for cx in (0, 1):
        ix = i1[:, 0] if cx else i0[:, 0]
        wx = t[:, 0] if cx else 1 - t[:, 0]
        for cy in (0, 1):
            iy = i1[:, 1] if cy else i0[:, 1]
            wy = t[:, 1] if cy else 1 - t[:, 1]
            for cz in (0, 1):
                iz = i1[:, 2] if cz else i0[:, 2]
                wz = t[:, 2] if cz else 1 - t[:, 2]
                out += (wx * wy * wz)[:, None] * flat[:, (ix * ng + iy) * ng + iz].T
    return out


def _rsd_device(x, v, f, obs):
    import torch
    d = x - obs
    rh = d / torch.linalg.norm(d, dim=1, keepdim=True).clamp_min(1e-30)
    return x + f * (v * rh).sum(1, keepdim=True) * rh


def batch_mock_device(n_mesh: int, n_gal: int, ran_ratio: int, b: float, f: float, shell: bool, seed: int,
                      device: str = "cuda", L: float | None = None) -> dict:
    """One mock of the batched workload on the GPU.  Box L = 6.84 N Mpc/h (the 512^3 survey's cell
    size) unless given, R = 15 Mpc/h.  Shell: observer at the centre of the x = 0 face, comoving 1100-1800 Mpc/h
    scaled by L/3500, 25% sky cap about +x, randoms ran_ratio x n_gal uniform in the window, mean
    density from the randoms.  Periodic: observer 1.5 L along -x of the box centre, uniform mean
    density (no randoms).  Returns params and float64 device positions."""
    import torch
    L = 6.84 * n_mesh if L is None else L
    gen = torch.Generator(device=device).manual_seed(seed)
    ng = min(n_mesh, 256)
    F = _field_device(ng, L, gen, device)
    if shell:
        sc = L / 3500.0
        r_min, r_max, cos_min = 1100.0 * sc, 1800.0 * sc, 0.5
        obs = torch.tensor([0.0, L / 2, L / 2], device=device, dtype=torch.float64)
        lo = torch.tensor([r_min * cos_min - 80.0, L / 2 - r_max - 80.0, L / 2 - r_max - 80.0],
                          device=device, dtype=torch.float64).clamp(0.0, L)
        hi = torch.tensor([r_max + 80.0, L / 2 + r_max + 80.0, L / 2 + r_max + 80.0],
                          device=device, dtype=torch.float64).clamp(0.0, L)
        vol_win = 0.25 * 4.0 / 3.0 * np.pi * (r_max ** 3 - r_min ** 3)
        per = int(n_gal * 2.0 * float(torch.prod(hi - lo)) / vol_win) + 1000
    else:
        obs = torch.tensor([L / 2 - 1.5 * L, L / 2, L / 2], device=device, dtype=torch.float64)
        lo = torch.zeros(3, device=device, dtype=torch.float64)
        hi = torch.full((3,), L, device=device, dtype=torch.float64)
        per = 2 * n_gal
    got, parts = 0, []
    while got < n_gal:
        q = lo + torch.rand((per, 3), generator=gen, device=device, dtype=torch.float64) * (hi - lo)
        s_ = _trilinear_device(F, q, L)
        keep = torch.rand(per, generator=gen, device=device) * 4.0 < torch.clamp(1.0 + (b - 1.0) * s_[:, 0], min=0.0)
        q, v = q[keep], s_[keep, 1:].double()
        s = _rsd_device(q + v, v, f, obs)
        if shell:
            d = s - obs
            r = torch.linalg.norm(d, dim=1)
            s = s[(r >= r_min) & (r <= r_max) & (d[:, 0] >= cos_min * r)]
        else:
            s = torch.remainder(s, L)
        parts.append(s)
        got += len(s)
    gal = torch.cat(parts)[:n_gal].contiguous()
    ran = None
    if shell:
        n_ran = n_gal * ran_ratio
        u = torch.rand((n_ran, 3), generator=gen, device=device, dtype=torch.float64)
        r = torch.pow(u[:, 0] * (r_max ** 3 - r_min ** 3) + r_min ** 3, 1.0 / 3.0)
        ct = cos_min + u[:, 1] * (1.0 - cos_min)
        st = torch.sqrt(torch.clamp(1 - ct * ct, min=0.0))
        ph = 2 * np.pi * u[:, 2]
        ran = obs + r[:, None] * torch.stack([ct, st * torch.cos(ph), st * torch.sin(ph)], 1)
        ran = ran.contiguous()
    params = dict(n=n_mesh, L=L, b=b, f=f, R=15.0, observer=tuple(float(v) for v in obs.cpu()), los_mode=0,
                  periodic=not shell, uniform=not shell, mask_frac=0.01, lognormal=False)
    return dict(params=params, gal=gal, ran=ran)


def batch_workload_device(count: int = 64, seed: int = 100, device: str = "cuda") -> list:
    """The batched workload: `count` mocks with N drawn from {256, 384, 512}, galaxies uniform in
    [2e5, 1e6], randoms 30-50 x galaxies, b in [1.5, 2.5], f in [0.6, 0.8]; even-numbered mocks are
    shell surveys and odd ones periodic boxes.  Mock i uses seed + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([256, 384, 512]))
        ng = int(rng.integers(200_000, 1_000_001))
        ratio = int(rng.integers(30, 51))
        b = float(rng.uniform(1.5, 2.5))
        f = float(rng.uniform(0.6, 0.8))
        out.append(batch_mock_device(n, ng, ratio, b, f, i % 2 == 0, seed + i, device))
    return out
