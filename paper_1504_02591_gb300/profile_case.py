"""Lean cases for kernel captures with ncu.

Default: the 512^3 mesh of the benchmark, a periodic box with uniform mean density and 2e5
galaxies (about 3 GB on the device), the iteration run by the host loop so that every pass is a
separately named kernel launch.

    python -m paper_1504_02591_gb300.profile_case --mesh 512 --iters 3 --repeat 2

--sort-tracers M: the brick sort and sorted deposit alone, M uniform float64 positions on the mesh
(3e7 on a 256^3 mesh is the benchmark's random catalogue in about 2.5 GB), deposited --repeat times;
with --shift, then one update and --repeat sorted shifts of the same tracers (the retained sort).

    python -m paper_1504_02591_gb300.profile_case --mesh 256 --sort-tracers 30000000 --repeat 3
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", type=int, default=512)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--sort-tracers", type=int, default=0)
    ap.add_argument("--shift", action="store_true")
    args = ap.parse_args(argv)
    import torch

    from . import binding as B
    from . import mocks
    if args.sort_tracers > 0:
        import numpy as np
        L = 3500.0
        m = mocks.periodic_box(L, args.mesh, 10_000, 0, 1.85, 0.74, 15.0, (0.0, L / 2, L / 2), 1, 2, 3, ng=64,
                               uniform=True)
        pos = torch.from_numpy(np.random.default_rng(7).uniform(0.0, L, (args.sort_tracers, 3))).cuda()
        r = B.Recon.from_mock(m, uniform=True)
        r.set_option(B.OPT_DEPOSIT_PATH, B.PATH_SORTED)
        for _ in range(args.repeat):
            r.deposit(pos, None, None, None)
        if args.shift:
            r.set_option(B.OPT_SHIFT_PATH, B.PATH_SORTED)
            r.set_option(B.OPT_REUSE_SORT, 1)
            r.smooth()
            r.iterate(B.START_FFTA, 0.0, 1)
            for _ in range(args.repeat):
                r.shift(pos, False)
        torch.cuda.synchronize()
        print("ok", args.sort_tracers)
        r.close()
        return
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
