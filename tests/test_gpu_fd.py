"""The finite-difference method of Sec. 2.1 (Eq. mainpot) on the GPU against the FP64 oracle.

The GPU solves A phi = delta/b with BiCGStab (float32 vectors, float64 inner products) preconditioned
by the FFT inverse of the periodic Laplacian; the oracle with GMRES in float64.  Both take the GPU's
smoothed delta, so the comparison isolates the operator, the solver and the gradient.  Tolerance:
rel L2 of Psi <= 1e-5 (the float32 vectors carry about 1e-7 relative rounding)."""
import numpy as np
import pytest

from oracle import recon_oracle as O
from paper_1504_02591_gb300 import mocks
from parity_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("los", ["radial", "fixed"])
def test_fd_solve_vs_oracle(lib, los):
    from paper_1504_02591_gb300 import binding as B
    m = mocks.scaled_shell(64, 6.84 * 64, 6_000, 40, 1.9, 0.74, 61)
    over = {} if los == "radial" else dict(los_mode=O.LOS_FIXED, observer=(0.8, 0.6, 0.0))
    p = m.params(**over)
    r = B.Recon.from_mock(m, **over)
    r.deposit(torch.from_numpy(m.galaxies.pos).cuda(), None, torch.from_numpy(m.randoms.pos).cuda(), None)
    r.smooth()
    delta = r.get_field(B.FIELD_DELTA).cpu().numpy().astype(np.float64)
    psi, it, res, st = r.fd_solve(tol=1e-7, max_iter=300)
    # the reconstruction proper still runs on the same handle afterwards
    n_it, rel, st2 = r.iterate(B.START_FFTA, 0.0, 3)
    assert n_it == 3
    r.close()
    want, phi, it_o, res_o = O.fd_solve(delta, p["b"], p["f"], p["L"], p["observer"], p["los_mode"], tol=1e-12)
    e = rel_l2(psi.cpu().numpy(), want)
    print(f"FD {los}: GPU {it} iterations, true residual {res:.1e}; oracle {it_o} GMRES iterations "
          f"(residual {res_o:.1e}); Psi rel L2 {e:.2e}")
    # the true residual of a float32 phi bottoms out near 1e-5: grid-scale rounding of phi, times the
    # Laplacian's 12 / g^2, against |A phi| of a field smooth over a few cells
    assert st == B.OK and res < 1e-4
    assert e <= 1e-5
