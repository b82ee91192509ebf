"""Shared helpers of the GPU parity tests (comparison metrics and the survey-mask tie rule)."""
import numpy as np

from oracle import recon_oracle as O

MASK_BAND = 1e-5   # relative distance to the mask threshold within which either decision is valid


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def mask_flips(ref, gpu_delta):
    """Flat indices where the GPU's survey mask (delta != 0) differs from the oracle's; asserts that
    each lies within rounding of the threshold (both decisions valid there)."""
    gd = gpu_delta.reshape(-1)
    omask = ref["mask"].reshape(-1)
    gmask = gd != 0
    # inside the mask delta itself can round to exactly 0 in float32 (rho_g = alpha rho_r to 24
    # bits): a zero where the oracle's delta is ~0 is no mask difference
    gmask |= (gd == 0) & omask & (np.abs(ref["delta"].reshape(-1)) < 1e-5)
    diff = np.nonzero(gmask != omask)[0]
    rr = ref["rho_r_s"].reshape(-1)[diff]
    thr = ref["threshold"]
    detail = [(int(i), float(v), float((v - thr) / thr), bool(gmask[i]), float(gd[i]))
              for i, v in zip(diff[:8], rr[:8])]
    assert np.all(np.abs(rr - thr) <= MASK_BAND * thr), \
        f"{len(diff)} mask differences, not all at the threshold {thr}: (node, rho_r_s, rel. distance, " \
        f"GPU in mask, GPU delta) {detail}"
    return diff


def reconstruct_same_branch(m, ref, gpu_delta, **kw):
    """The oracle rerun with the GPU's decisions at the mask ties (each a valid branch)."""
    diff = mask_flips(ref, gpu_delta)
    if len(diff) == 0:
        return ref
    return O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos, None, mask_flip=diff, **kw)


def host_mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0
