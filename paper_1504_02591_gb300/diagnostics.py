"""Host-side rules of the paper's diagnostics (the statistics themselves run on the GPU through
recon_radial_ratio, recon_ratio_stats and recon_helmholtz_x)."""
from __future__ import annotations


def converged_at(means, tol: float = 0.01) -> int:
    """Sec. 5.2 (captions of Tables 2 and 3): the iteration from which on the mean radial ratio
    changes by no more than tol between consecutive iterations, |m[k+1] - m[k]| <= tol for every
    k >= n; the last iteration when no earlier one qualifies.  The ratios sit near 1, so the
    paper's 1% is an absolute 0.01, and the bound is inclusive: the paper's printed two-decimal
    tables then give the iteration counts it states (4 and 2 in Table 2, 6 and 2 in Table 3)."""
    m = [float(x) for x in means]
    if not m:
        raise ValueError("no means")
    n = len(m) - 1
    # walk back from the end while the step into the current iteration stays within tol
    while n > 0 and abs(m[n] - m[n - 1]) <= tol + 1e-12:
        n -= 1
    return n
