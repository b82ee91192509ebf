"""recon_cic_deposit_noalloc: the deposit entry point for callers that cannot allocate device memory.

Such callers (plugins whose host owns all device memory, real-time pipelines that must not enter an
allocator) get a CIC deposit whose only scratch is a fixed array inside the library.  This test
calls it through the C ABI twice in a row and checks each result against the ordinary handle-based
deposit (recon_deposit) on the same catalogue, and against the FP64 oracle's CIC deposit and a
float64 sum of the weights.  The file is named to be collected last, so a stop at the first failure
has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import recon_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, L = 64, 1000.0


def reference_deposit(B, pos, w):
    """The existing entry point: a handle in uniform mode deposits the catalogue as galaxies."""
    r = B.Recon(N, L, 2.0, 0.7, 10.0, (0, 0, 0), uniform=True)
    r.deposit(pos, w, None, None)
    rho = r.get_field(B.FIELD_RHO_G).clone()
    sw = r.scalars()["sum_wg"]
    r.close()
    return rho, sw


def noalloc_deposit(lib, B, pos, w, rho, sum_w):
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.recon_cic_deposit_noalloc(C.c_void_p(pos.data_ptr()), B.F64 if pos.dtype == torch.float64 else B.F32,
                                       C.c_void_p(w.data_ptr()) if w is not None else None, pos.shape[0], N, L,
                                       C.c_void_p(rho.data_ptr()), C.c_void_p(sum_w.data_ptr()),
                                       C.c_void_p(stream))
    assert st == B.OK, lib.recon_status_str(st)
    torch.cuda.synchronize()


def test_noalloc_deposit_matches_handle_deposit_twice(lib):
    from paper_1504_02591_gb300 import binding as B
    rng = np.random.default_rng(2024)
    rho = torch.empty((N, N, N), dtype=torch.float32, device="cuda")      # caller-owned outputs
    sum_w = torch.empty(1, dtype=torch.float64, device="cuda")
    cases = [
        (torch.from_numpy(rng.uniform(0, L, (300_001, 3))).cuda(), None),
        (torch.from_numpy(rng.uniform(0, L, (123_457, 3)).astype(np.float32)).cuda(),
         torch.from_numpy(rng.uniform(0.5, 2.0, 123_457).astype(np.float32)).cuda()),
    ]
    for pos, w in cases:                       # two calls in a row on the shared scratch
        noalloc_deposit(lib, B, pos, w, rho, sum_w)
        want_rho, want_sw = reference_deposit(B, pos, w)
        got = rho.double()
        err = float(((got - want_rho.double()) ** 2).sum().sqrt() / (want_rho.double() ** 2).sum().sqrt())
        assert err < 1e-6, err
        assert float(sum_w.item()) == pytest.approx(want_sw, rel=1e-12)
        # and the FP64 oracle (Sec. 3 binning with the CIC kernel), weights summed in float64
        pos64 = pos.cpu().numpy().astype(np.float64)
        w64 = None if w is None else w.cpu().numpy().astype(np.float64)
        ref = O.cic_deposit(pos64, w64, N, L)
        err_o = float(np.sqrt(((got.cpu().numpy() - ref) ** 2).sum() / (ref ** 2).sum()))
        assert err_o < 1e-6, err_o
        want_w = float(len(pos64)) if w64 is None else float(w64.sum())
        assert float(sum_w.item()) == pytest.approx(want_w, rel=1e-12)


def test_noalloc_rejects_too_many_particles(lib):
    from paper_1504_02591_gb300 import binding as B
    rho = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    sum_w = torch.empty(1, dtype=torch.float64, device="cuda")
    dummy = torch.empty((1, 3), dtype=torch.float64, device="cuda")
    st = lib.recon_cic_deposit_noalloc(C.c_void_p(dummy.data_ptr()), B.F64, None, 67_108_864 + 1, N, L,
                                       C.c_void_p(rho.data_ptr()), C.c_void_p(sum_w.data_ptr()), None)
    assert st == B.ERR_INVALID_ARG
