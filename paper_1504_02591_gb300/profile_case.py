"""A lean reconstruction for kernel captures with ncu: the 512^3 mesh of the benchmark, a periodic
box with uniform mean density and 2e5 galaxies (about 3 GB on the device), the iteration run by
the host loop so that every pass is a separately named kernel launch.

    python -m paper_1504_02591_gb300.profile_case --mesh 512 --iters 3 --repeat 2
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", type=int, default=512)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args(argv)
    import torch

    from . import binding as B
    from . import mocks
    L = 3500.0 * args.mesh / 512
    m = mocks.periodic_box(L, args.mesh, 200_000, 0, 1.85, 0.74, 15.0, (0.0, L / 2, L / 2), 1, 2, 3, ng=128,
                           uniform=True)
    r = B.Recon.from_mock(m, uniform=True)
    r.set_option(B.OPT_GRAPH, 0)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    for _ in range(args.repeat):
        r.deposit(gal, None, None, None)
        r.smooth()
        n, rel, st = r.iterate(B.START_FFTA, 0.0, args.iters)
    torch.cuda.synchronize()
    print("ok", n, rel)
    r.close()


if __name__ == "__main__":
    main()
