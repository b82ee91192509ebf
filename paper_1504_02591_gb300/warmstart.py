"""Learned warm start: training pairs from the method itself, training, and the warm-started solve.

Everything numerical runs in the library's CUDA kernels (recon_* and recon_unet_*); this module only
sequences the calls.  The network maps (delta, r, u_0) -> u, where u_0 = Psi_0 . r is the radial
displacement of the Eq. approx2 start and u = Psi . r that of the converged solution of Eq. Nusser;
the iteration then runs from P_0 = u r to the usual stopping rule, so the network can only change
how many updates are needed, not the answer.
"""
from __future__ import annotations

import os

import numpy as np

from . import binding as B


def training_pair(mock, level=0, tol=1e-6, max_iter=120, start=B.START_FFTA):
    """(features, target, n_iter) for one mock: the network inputs after smoothing and the block means
    of the converged radial displacement from the plain method (the iteration from the analytic
    start), both on the mesh coarsened `level` times."""
    r = B.Recon.from_mock(mock)
    try:
        r.deposit(mock.galaxies.pos, None, None if mock.randoms is None else mock.randoms.pos, None)
        r.smooth()
        feat = r.start_features(start, level)
        n_it, rel, st = r.iterate(start, tol, max_iter)
        u = r.get_radial(level)
    finally:
        r.close()
    return feat, u, n_it


def train(net, pairs, steps, lr=1e-3, wd=1e-4, warmup=20):
    """AdamW on the mean squared error of u over the pairs (round robin); returns the losses."""
    losses = []
    for s in range(steps):
        feat, u = pairs[s % len(pairs)][:2]
        losses.append(net.backward(feat, u))
        scale = min(1.0, (s + 1) / warmup)
        net.adamw(lr * scale, wd)
    return losses


def warm_iterate(recon, net, level=0, tol=1e-6, max_iter=120):
    """After recon.smooth(): network start on the mesh coarsened `level` times, then the iteration
    to the stopping rule."""
    feat = recon.start_features(B.START_FFTA, level)
    u0 = net.forward(feat)
    return recon.iterate_from(u0, tol, max_iter, level)


def save(net, path, level, meta=None):
    """Weights (float32, the ABI's parameter order), width, level; meta (a dict) as JSON beside."""
    import json
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez(path, params=net.get_params(), c1=net.c1, level=level)
    if meta is not None:
        with open(os.path.splitext(path)[0] + ".json", "w") as f:
            json.dump(meta, f, indent=1)


def load(path, bf16=True):
    """(network, level) from a file written by save()."""
    d = np.load(path)
    net = B.UNet(c1=int(d["c1"]), bf16=bf16)
    net.set_params(d["params"])
    return net, int(d["level"])


def default_weights_path():
    """The network trained for the 512^3 survey-shell workload (train_warmstart.py)."""
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warm_shell512_c8_l2.npz")
