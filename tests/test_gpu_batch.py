"""Batched reconstruction (recon_batch_run): mixed mesh sizes, windows and parameters in one call.

Every item must give the same result as the same mock reconstructed alone through the handle API
(up to float32 summation order), and one item is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import recon_oracle as O
from paper_1504_02591_gb300 import mocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch_mocks():
    ms = [
        mocks.periodic_box(1000.0, 32, 20_000, 200_000, 2.0, 0.74, 15.0, (2000.0, 500.0, 500.0), 1, 2, 3, ng=64),
        mocks.scaled_shell(64, 1000.0, 20_000, 30, 1.6, 0.65, 40),
        mocks.periodic_box(800.0, 48, 30_000, 300_000, 2.4, 0.8, 15.0, (-300.0, 400.0, 400.0), 4, 5, 6, ng=48),
        mocks.scaled_shell(64, 1200.0, 25_000, 40, 2.2, 0.7, 50),
        mocks.periodic_box(1000.0, 32, 15_000, 150_000, 1.5, 0.6, 15.0, (1.0, 0.0, 0.0), 7, 8, 9, ng=64, los_mode=1),
    ]
    return ms


def test_batch_matches_single_runs(lib, batch_mocks):
    from paper_1504_02591_gb300 import binding as B
    status, res = B.batch_run(batch_mocks, start=B.START_FFTA, tol=1e-6, max_iter=60)
    assert status == B.OK
    for n in (32, 48, 64):
        assert B.batch_plan(n) is not None
    for m, r in zip(batch_mocks, res):
        assert r["status"] in (B.OK, B.ERR_NOT_CONVERGED) and r["ms"] > 0
        single = B.Recon.from_mock(m)
        gal = torch.from_numpy(m.galaxies.pos).cuda()
        ran = torch.from_numpy(m.randoms.pos).cuda()
        n_it, rel, st = single.run(gal, ran, start=B.START_FFTA, tol=1e-6, max_iter=60)
        assert abs(n_it - r["n_iter"]) <= 1
        sg = single.shift(gal, True).cpu().numpy()
        sr = single.shift(ran, False).cpu().numpy()
        single.close()
        assert np.abs(r["shift_gal"].cpu().numpy() - sg).max() <= 1e-4
        assert np.abs(r["shift_ran"].cpu().numpy() - sr).max() <= 1e-4


def test_batch_one_graph_matches(lib, batch_mocks):
    """RECON_BATCH_ONE_GRAPH (the whole batch as one graph, size classes side by side) gives the same
    reconstructions as the per-mock graphs launched back to back (up to the float32 order of the
    deposit atomics)."""
    from paper_1504_02591_gb300 import binding as B
    s0, r0 = B.batch_run(batch_mocks, start=B.START_FFTA, tol=1e-6, max_iter=60)
    s1, r1 = B.batch_run(batch_mocks, start=B.START_FFTA, tol=1e-6, max_iter=60, one_graph=True)
    assert s0 == B.OK and s1 == B.OK
    for a, b in zip(r0, r1):
        assert b["status"] == a["status"] and abs(a["n_iter"] - b["n_iter"]) <= 1 and b["ms"] > 0
        assert np.abs(a["shift_gal"].cpu().numpy() - b["shift_gal"].cpu().numpy()).max() <= 1e-4
        assert np.abs(a["shift_ran"].cpu().numpy() - b["shift_ran"].cpu().numpy()).max() <= 1e-4
    # the shifts written into the caller's buffers of an earlier call
    bufs = [(torch.full_like(a["shift_gal"], float("nan")), torch.full_like(a["shift_ran"], float("nan")))
            for a in r0]
    s2, r2 = B.batch_run(batch_mocks, start=B.START_FFTA, tol=1e-6, max_iter=60, out=bufs)
    assert s2 == B.OK
    for (bg, br), a, c in zip(bufs, r1, r2):
        assert c["shift_gal"] is bg and c["shift_ran"] is br
        assert np.abs(a["shift_gal"].cpu().numpy() - bg.cpu().numpy()).max() <= 1e-4
        assert np.abs(a["shift_ran"].cpu().numpy() - br.cpu().numpy()).max() <= 1e-4


def test_batch_item_vs_oracle(lib, batch_mocks):
    from paper_1504_02591_gb300 import binding as B
    m = batch_mocks[0]
    status, res = B.batch_run([m], start=B.START_PLAIN, tol=0.0, max_iter=6)
    assert status == B.OK and res[0]["n_iter"] == 6
    ref = O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos, None, start=O.START_PLAIN, tol=0.0,
                        max_iter=6)
    assert np.abs(res[0]["shift_gal"].cpu().numpy() - ref["shift_g"]).max() <= 1e-4
    assert np.abs(res[0]["shift_ran"].cpu().numpy() - ref["shift_r"]).max() <= 1e-4


def test_batch_rejects_bad_item(lib, batch_mocks):
    """An unsupported mesh in one item fails that item only; the others still run."""
    from paper_1504_02591_gb300 import binding as B
    import ctypes as C
    m = batch_mocks[0]
    items = (B.ReconBatchItem * 2)()
    keep = []
    for i, n in enumerate((32, 100)):
        p = m.params()
        items[i].params = B.make_params(n, p["L"], p["b"], p["f"], p["R"], p["observer"])
        g = torch.from_numpy(m.galaxies.pos).cuda()
        r = torch.from_numpy(m.randoms.pos).cuda()
        items[i].gal = B._catalog(g, None, keep)
        items[i].ran = B._catalog(r, None, keep)
        items[i].start, items[i].tol, items[i].max_iter, items[i].out_on_device = 0, 0.0, 3, 1
    st = lib.recon_batch_run(items, 2, C.c_void_p(torch.cuda.current_stream().cuda_stream), 0)
    assert st == B.ERR_INVALID_ARG
    assert items[0].status == B.OK and items[0].n_iter == 3
    assert items[1].status == B.ERR_INVALID_ARG


def test_batch_384_item_vs_oracle(lib):
    """A 384^3 survey shell (one of the batched workload's mesh sides) reconstructed inside a batch
    graph next to a 256^3 periodic box: its shifts equal the FP64 oracle's for the same 3 updates."""
    from paper_1504_02591_gb300 import binding as B
    m = mocks.scaled_shell(384, 6.84 * 384, 200_000, 30, 2.1, 0.65, 140)
    other = mocks.batch_mock_device(256, 200_000, 30, 1.7, 0.7, False, 7)
    status, res = B.batch_run([other, m], start=B.START_FFTA, tol=0.0, max_iter=3)
    assert status == B.OK and res[1]["n_iter"] == 3 and res[0]["n_iter"] == 3
    ref = O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos, None, start=O.START_FFTA, tol=0.0,
                        max_iter=3, shift=False)
    p = m.params()
    rng = np.random.default_rng(5)
    ir = rng.choice(len(m.randoms.pos), 200_000, replace=False)
    dg = O.shift_vectors(ref["psi"], m.galaxies.pos, p["L"], p["f"], p["observer"], p["los_mode"], True)
    dr = O.shift_vectors(ref["psi"], m.randoms.pos[ir], p["L"], p["f"], p["observer"], p["los_mode"], False)
    e_g = float(np.abs(res[1]["shift_gal"].cpu().numpy() - dg).max())
    e_r = float(np.abs(res[1]["shift_ran"].cpu().numpy()[ir] - dr).max())
    print(f"batch 384^3 item: shifts {e_g:.2e} / {e_r:.2e} Mpc/h, {res[1]['ms']:.2f} ms")
    assert e_g <= 1e-4 and e_r <= 1e-4
