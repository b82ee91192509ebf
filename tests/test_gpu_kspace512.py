"""The register-fused source-update kernel (N = 512) against the generic staged kernel.

Both compute every butterfly with the same operations in the same order, so after a fixed number of
updates Psi is identical bit for bit; only the order of the float32 norm sums differs.  The generic
kernel is checked against the FP64 oracle at the smaller meshes of test_gpu_parity.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("los_mode", [0, 1])
def test_fused_kspace_kernel_matches_generic(lib, los_mode):
    """The whole update (y pass, paired x passes, z pass with the two-field vector forms) fused
    against generic, for a radial and a fixed line of sight (the z pass's two forms of d and w)."""
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import mocks
    m = mocks.periodic_box(3500.0, 512, 100_000, 0, 1.85, 0.74, 15.0, (0.0, 1750.0, 1750.0), 4, 5, 6, ng=128,
                           los_mode=los_mode, uniform=True)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    r = B.Recon.from_mock(m, uniform=True)
    out = {}
    # one deposit (its float atomics make the mesh differ in the last bits from run to run), two
    # iterations on the same delta(k)
    r.deposit(gal, None, None, None)
    r.smooth()
    for generic in (1, 0):
        r.set_option(B.OPT_KSPACE_GENERIC, generic)
        n, rel, st = r.iterate(B.START_FFTA, 0.0, 4)
        out[generic] = (r.get_psi().cpu().numpy(), np.array(r.trace()))
    r.close()
    psi_g, tr_g = out[1]
    psi_f, tr_f = out[0]
    d = float(np.sqrt(((psi_f.astype(np.float64) - psi_g) ** 2).sum() / (psi_g.astype(np.float64) ** 2).sum()))
    print(f"fused vs generic: rel L2 of Psi {d:.2e}, bitwise equal: {np.array_equal(psi_f, psi_g)}")
    # the same butterflies; any difference is the compiler's contraction of a product and a sum
    # into one fused multiply-add, a float32 rounding per operation
    assert d < 1e-6
    assert np.allclose(tr_f, tr_g, rtol=1e-4, atol=0)


def test_fused_warm_start_passes_512(lib):
    """At N = 512 the warm start's Z passes run fused too: a zero correction still reproduces the
    Eq. approx2 iteration bit for bit, and a non-zero correction agrees with the generic passes."""
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import mocks
    m = mocks.periodic_box(3500.0, 512, 100_000, 0, 1.85, 0.74, 15.0, (0.0, 1750.0, 1750.0), 7, 8, 9, ng=128,
                           uniform=True)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    r = B.Recon.from_mock(m, uniform=True)
    r.deposit(gal, None, None, None)
    r.smooth()
    feat = r.start_features(B.START_FFTA, 2)
    r.iterate_from(feat[..., 4].contiguous(), 0.0, 3, 2)
    psi_w, tr_w = r.get_psi().cpu().numpy(), r.trace()
    r.iterate(B.START_FFTA, 0.0, 3)
    psi_a, tr_a = r.get_psi().cpu().numpy(), r.trace()
    assert tr_w == tr_a and np.array_equal(psi_w, psi_a)
    g = torch.Generator().manual_seed(5)
    noise = 0.5 * torch.randn((128, 128, 128), generator=g).cuda()
    out = {}
    for generic in (1, 0):
        r.set_option(B.OPT_KSPACE_GENERIC, generic)
        r.deposit(gal, None, None, None)   # the iteration reused the density fields: deposit again
        r.smooth()
        feat = r.start_features(B.START_FFTA, 2)
        r.iterate_from((feat[..., 4] + noise).contiguous(), 0.0, 3, 2)
        out[generic] = r.get_psi().cpu().numpy()
    r.close()
    d = float(np.sqrt(((out[0].astype(np.float64) - out[1]) ** 2).sum() / (out[1].astype(np.float64) ** 2).sum()))
    # the two deposits differ in the order of their float32 atomic sums (about 1e-7)
    assert d < 1e-6, d


@pytest.mark.parametrize("uniform", [False, True])
def test_fused_delta_pass_512(lib, uniform):
    """The z convolution, delta and its r2c at N = 512, and the start's y pass (delta(k), S_-1 and
    Z[delta/b]), fused against generic: the real delta, delta(k) and Psi after one update agree up
    to the order of the deposit's float32 atomic sums."""
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import mocks
    if uniform:
        m = mocks.periodic_box(3500.0, 512, 100_000, 0, 1.85, 0.74, 15.0, (0.0, 1750.0, 1750.0), 4, 5, 6, ng=128,
                               uniform=True)
    else:
        m = mocks.survey_shell_512(n_gal=100_000, ran_ratio=20)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = None if uniform else torch.from_numpy(m.randoms.pos).cuda()
    r = B.Recon.from_mock(m, uniform=uniform)
    out = {}
    for generic in (1, 0):
        r.set_option(B.OPT_KSPACE_GENERIC, generic)
        r.deposit(gal, None, ran, None)
        r.smooth()
        d_real = r.get_field(B.FIELD_DELTA).cpu().numpy()
        r.iterate(B.START_FFTA, 0.0, 1)          # delta(k) is exported once the y transform has run
        out[generic] = (d_real, r.get_field(B.FIELD_DELTA_K).cpu().numpy(), r.get_psi().cpu().numpy())
    r.close()
    for i in range(3):
        dt = np.complex128 if np.iscomplexobj(out[0][i]) else np.float64
        a, b = out[0][i].astype(dt), out[1][i].astype(dt)
        d = float(np.sqrt((np.abs(a - b) ** 2).sum() / (np.abs(b) ** 2).sum()))
        print(f"fused delta pass ({'uniform' if uniform else 'survey'}), {('delta', 'delta(k)', 'Psi')[i]}: rel L2 {d:.2e}")
        assert d < 1e-5, d


def test_narrow_line_tiles_512(lib):
    """RECON_OPT_LINE_TILE = 1 (8-column x tiles, also for the paired vector x passes) gives the
    update of the default 16-column tiles: the same butterflies on the same columns."""
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import mocks
    m = mocks.periodic_box(3500.0, 512, 100_000, 0, 1.85, 0.74, 15.0, (0.0, 1750.0, 1750.0), 4, 5, 6, ng=128,
                           uniform=True)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    r = B.Recon.from_mock(m, uniform=True)
    r.deposit(gal, None, None, None)
    r.smooth()
    out = {}
    for tile in (0, 1):
        r.set_option(B.OPT_LINE_TILE, tile)
        r.iterate(B.START_FFTA, 0.0, 4)
        out[tile] = r.get_psi().cpu().numpy().astype(np.float64)
    r.close()
    d = float(np.sqrt(((out[1] - out[0]) ** 2).sum() / (out[0] ** 2).sum()))
    assert d < 1e-6, d


@pytest.mark.parametrize("graph", [1, 0])
def test_plane_batched_passes_match_unbatched(lib, graph):
    """RECON_OPT_PLANE_BATCH runs the same kernels on the same elements, only grouped by y-planes
    (x inverse, projection and x forward per batch), so Psi and the trace are bitwise those of the
    unbatched passes, in the device-driven graph loop and in the host-driven loop, for every batch
    size; with a tolerance the stopping update is the same too."""
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import mocks
    m = mocks.periodic_box(3500.0, 512, 100_000, 0, 1.85, 0.74, 15.0, (0.0, 1750.0, 1750.0), 4, 5, 6, ng=128,
                           uniform=True)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    r = B.Recon.from_mock(m, uniform=True)
    r.set_option(B.OPT_GRAPH, graph)
    r.deposit(gal, None, None, None)
    r.smooth()
    out = {}
    for planes in (0, 16, 32, 64):
        r.set_option(B.OPT_PLANE_BATCH, planes)
        n, rel, st = r.iterate(B.START_FFTA, 0.0, 4)
        out[planes] = (r.get_psi().cpu().numpy(), np.array(r.trace()))
        n_c, rel_c, st_c = r.iterate(B.START_FFTA, 1e-6, 40)
        out[planes] += (n_c, r.get_psi().cpu().numpy())
    r.close()
    for planes in (16, 32, 64):
        assert np.array_equal(out[planes][0], out[0][0]), planes
        assert np.array_equal(out[planes][1], out[0][1]), planes
        assert out[planes][2] == out[0][2] and np.array_equal(out[planes][3], out[0][3]), planes


@pytest.mark.parametrize("los_mode", [0, 1])
def test_tma_streamed_update_matches_direct_loads(lib, los_mode):
    """RECON_OPT_KITER_TMA: the source update with its inputs streamed into shared memory by the
    tensor memory accelerator (persistent CTAs) computes every element with the same arithmetic as
    the one-tile-per-CTA kernel, so Psi after a fixed number of updates is bitwise equal; its threads
    accumulate the norm sums in float32 over several tiles, so the trace agrees to float32 rounding."""
    from paper_1504_02591_gb300 import binding as B
    from paper_1504_02591_gb300 import mocks
    obs = (0.0, 1750.0, 1750.0) if los_mode == 0 else (0.6, 0.8, 0.0)
    m = mocks.periodic_box(3500.0, 512, 100_000, 0, 1.85, 0.74, 15.0, obs, 4, 5, 6, ng=128,
                           los_mode=los_mode, uniform=True)
    r = B.Recon.from_mock(m, uniform=True)
    r.deposit(torch.from_numpy(m.galaxies.pos).cuda(), None, None, None)
    r.smooth()
    out = {}
    for tma in (0, 1):
        r.set_option(B.OPT_KITER_TMA, tma)
        for graph in (1, 0):
            r.set_option(B.OPT_GRAPH, graph)
            n, rel, st = r.iterate(B.START_FFTA, 0.0, 5)
            out[(tma, graph)] = (r.get_psi().cpu().numpy(), np.array(r.trace()))
    r.close()
    base = out[(0, 1)]
    for key, (psi, tr) in out.items():
        assert np.array_equal(psi, base[0]), key
        assert np.allclose(tr, base[1], rtol=1e-5, atol=0), key
