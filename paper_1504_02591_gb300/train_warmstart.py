"""Train the learned warm start for the 512^3 survey-shell workload.

Pairs come from the plain method itself: for each synthetic survey mock (the benchmark's geometry
and statistics, other seeds), the library computes the network inputs on the mesh coarsened
`level` times (block means of delta, r and the Eq. approx2 start's radial displacement) and
iterates from the analytic start to 1e-6; the target is the block means of the converged Psi . r.
The U-Net is trained with the library's own forward, backward and AdamW kernels; the benchmark mock
(seed 10) is held out and evaluated at the end.  Runs on the GPU:

    python -m paper_1504_02591_gb300.train_warmstart --mocks 16 --steps 2000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as B
from . import mocks
from . import warmstart as W


def _init_params(c1, seed):
    """He-normal 3x3x3 weights, zero biases, zero head (the network starts as the analytic start)."""
    rng = np.random.default_rng(seed)
    parts = []
    c2, c3 = 2 * c1, 4 * c1
    specs = [(5, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3), (c3 + c2, c2), (c2, c2), (c2 + c1, c1),
             (c1, c1)]
    for ci, co in specs:
        parts += [rng.standard_normal(27 * ci * co) * np.sqrt(2.0 / (27 * ci)), np.zeros(co)]
    parts += [np.zeros(c1), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--mocks", type=int, default=16)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--level", type=int, default=2)
    ap.add_argument("--c1", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--wd", type=float, default=1e-4)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--out", default=W.default_weights_path())
    ap.add_argument("--device-mocks", action="store_true",
                    help="draw the training galaxies on the GPU (mocks.batch_mock_device, same recipe and "
                         "survey geometry), so hundreds of mocks take minutes")
    args = ap.parse_args(argv)
    import torch

    t0 = time.time()
    shared = mocks.survey_shell_512(seed=args.seed0 - 3)     # its randoms serve every training mock
    pairs, n_plain = [], []
    ran_dev = torch.from_numpy(shared.randoms.pos).cuda() if args.device_mocks else None
    for i in range(args.mocks):
        if args.device_mocks:
            d = mocks.batch_mock_device(512, 600_000, 0, shared.b, shared.f, True, args.seed0 + i, L=shared.L)
            m = mocks.Mock("shell-512-device", shared.L, 512, shared.b, shared.f, shared.R, shared.observer, 0, False,
                           False, galaxies=mocks.Catalog(d["gal"]), randoms=mocks.Catalog(ran_dev))
        else:
            m = shared if i == 0 else mocks.survey_shell_512(ran_ratio=0, seed=args.seed0 + 3 * i)
            m.randoms = shared.randoms
        feat, u, n_it = W.training_pair(m, args.level)
        pairs.append((feat, u))
        n_plain.append(n_it)
    t_pairs = time.time() - t0
    net = B.UNet(c1=args.c1, bf16=True)
    net.set_params(_init_params(args.c1, args.seed0))
    t1 = time.time()
    losses = W.train(net, pairs, steps=args.steps, lr=args.lr, wd=args.wd)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    del pairs

    # held-out evaluation on the benchmark mock
    m = mocks.survey_shell_512()
    feat, u_conv, n_ffta = W.training_pair(m, args.level)
    y = net.forward(feat)
    err_ffta = float(((feat[..., 4] - u_conv) ** 2).sum().sqrt() / (u_conv ** 2).sum().sqrt())
    err_net = float(((y - u_conv) ** 2).sum().sqrt() / (u_conv ** 2).sum().sqrt())
    r = B.Recon.from_mock(m)
    r.deposit(m.galaxies.pos, None, m.randoms.pos, None)
    r.smooth()
    n_warm, rel, st = W.warm_iterate(r, net, args.level, 1e-6, 120)
    r.close()
    seeds = ([args.seed0 + i for i in range(args.mocks)] if args.device_mocks else
             [args.seed0 - 3] + [args.seed0 + 3 * i for i in range(1, args.mocks)])
    meta = dict(workload="survey_shell_512", level=args.level, c1=args.c1, mocks=args.mocks, seed0=args.seed0,
                device_mocks=bool(args.device_mocks), seeds=seeds, steps=args.steps,
                lr=args.lr, wd=args.wd, loss_first=float(np.mean(losses[:20])), loss_last=float(np.mean(losses[-100:])),
                plain_updates_train=n_plain, heldout=dict(seed=10, start_error_ffta=err_ffta, start_error_learned=err_net,
                                                          updates_ffta=n_ffta, updates_learned=n_warm, rel=rel),
                seconds=dict(pairs=t_pairs, train=t_train))
    W.save(net, args.out, args.level, meta)
    net.close()
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
