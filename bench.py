#!/usr/bin/env python
"""Benchmark: milliseconds per converged 512^3 reconstruction on GB300.

One step = the whole path on one synthetic survey: CIC deposit of 6e5 galaxies and 3e7 randoms,
Gaussian smoothing and delta with the survey mask, the Fourier-space iteration until
|dPsi|/|Psi| < 1e-6 from the learned warm start (when its trained weights are present; the line also
reports the RSD-corrected Eq. approx2 start and the uncorrected one), and the shift of every galaxy
and random.  Inputs are resident in HBM when the timed region starts; every field (539 MB) is larger
than L2, so no explicit L2 flush is needed.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank reconstructs its own replica (the solve does not shard; the job
is a set of independent reconstructions), and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per converged 512^3 reconstruction, plain vs warm-start; % HBM peak"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--mesh", type=int, default=512)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=80)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-warm", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 1024^3 large periodic run")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT context timing")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-mock batch")
    ap.add_argument("--no-diag", action="store_true", help="skip the paper's diagnostics")
    ap.add_argument("--cpu-full", action="store_true",
                    help="only run the whole FP64 oracle on the result table's workloads (host cores)")
    ap.add_argument("--cpu-full-1024", action="store_true", help="with --cpu-full: also the 1024^3 run (~150 GB)")
    ap.add_argument("--plane-batch", type=int, default=None,
                    help="y-planes per batch of the x -> z -> x passes (0 off; default: the library's)")
    ap.add_argument("--particle-order", choices=("retained", "per-call"), default="retained",
                    help="retained: one brick sort per catalogue per step, shared by deposit and shift")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven iteration (every pass a plain launch; for ncu launch lists)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBps", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def workload(mesh):
    from paper_1504_02591_gb300 import mocks
    return mocks.survey_shell_512(n_mesh=mesh)


def workload_name(mesh):
    return (f"survey shell {mesh}^3, L=3500 Mpc/h, 6e5 galaxies + 3e7 randoms (50x), shell 1100-1800 "
            f"Mpc/h, 25% sky, b=1.85 f=0.74 R=15, converged to 1e-6")


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = [l.split(",") for l in open(self.tmp.name).read().strip().splitlines() if l.count(",") >= 8]
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if "Active" in r[5 + j] and "Not" not in r[5 + j]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, device):
    """The slowest rank's time, on every rank (unchanged without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_per_step, world_size):
    """Whole-job ms per converged reconstruction: every rank reconstructs its own mock per step
    (replicas), so N ranks finish N reconstructions in the slowest rank's step time."""
    return ms_per_step / world_size


RAN_SAMPLE = 3_000_000      # randoms deposited and shifted by the CPU sample (timing scales with count)


def oracle_stages(m, n_iter, cores):
    """The FP64 oracle as it stands, timed stage by stage on the full-size workload (512^3 mesh).

    Every mesh stage runs at full size: smoothing of both densities, delta with the survey mask,
    the line-of-sight field, the Eq. approx2 start and one update of Eq. iterative.  The particle
    stages (CIC deposit and shift) run on all galaxies and on RAN_SAMPLE of the randoms; their time
    is linear in the particle count and is scaled to all randoms.  A converged reconstruction is
    then deposit + smoothing + delta + start + n_iter updates + shift.  The library FFT runs on
    `cores` threads; numpy's elementwise work is single-threaded."""
    import numpy as np
    from oracle import recon_oracle as O
    O.FFT_WORKERS = cores
    O.fft3(np.zeros((32, 32, 32)))                     # the FFT's thread pool and plan cache
    p = m.params()
    n, L = p["n"], p["L"]
    gal, ran = m.galaxies.pos, m.randoms.pos
    rs = min(RAN_SAMPLE, len(ran))
    scale_r = len(ran) / rs
    t = {}
    c0 = time.perf_counter()
    t0 = time.perf_counter()
    rho_g = O.cic_deposit(gal, None, n, L)
    tg = time.perf_counter() - t0
    t0 = time.perf_counter()
    rho_r = O.cic_deposit(ran[:rs], None, n, L)
    t["deposit"] = tg + (time.perf_counter() - t0) * scale_r
    t0 = time.perf_counter()
    rho_g_s = O.smooth(rho_g, p["R"], L)
    rho_r_s = O.smooth(rho_r, p["R"], L)
    t["smooth"] = time.perf_counter() - t0
    rho_r_s *= scale_r                                 # the full random catalogue's density scale
    t0 = time.perf_counter()
    delta, _, _, _ = O.overdensity_randoms(rho_g_s, rho_r_s, float(len(gal)), float(len(ran)),
                                           p["mask_frac"], int(np.count_nonzero(rho_r > 0)))
    t["delta"] = time.perf_counter() - t0
    del rho_g, rho_r, rho_g_s, rho_r_s
    t0 = time.perf_counter()
    rhat = O.rhat_field(n, L, p["observer"], p["los_mode"])
    t["rhat"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    psi, _ = O.start_estimate(delta, p["b"], p["f"], L, rhat, O.START_FFTA)
    t["start"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    psi = O.update(psi, delta, p["b"], p["f"], L, rhat)
    t["update"] = time.perf_counter() - t0
    del rhat, delta
    t0 = time.perf_counter()
    O.shift_vectors(psi, gal, L, p["f"], p["observer"], p["los_mode"], True)
    tg = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.shift_vectors(psi, ran[:rs], L, p["f"], p["observer"], p["los_mode"], False)
    t["shift"] = tg + (time.perf_counter() - t0) * scale_r
    cpu_s = time.perf_counter() - c0
    total = sum(v for k, v in t.items() if k != "update") + n_iter * t["update"]
    return total * 1000.0, {k: round(v, 3) for k, v in t.items()}, cpu_s


def cpu_full(args):
    """The FP64 oracle as it stands, run whole (no sampling) on the workloads of the results table:
    the 64^3 periodic box (6 updates, uncorrected and Eq. approx2 starts), the 512^3 survey shell to
    1e-6, and the 1024^3 periodic box (6 updates) when the host has the memory; all host cores and
    one core.  Prints one JSON line per run."""
    import numpy as np
    from oracle import recon_oracle as O
    from paper_1504_02591_gb300 import mocks
    cores = os.cpu_count() or 1

    def run(name, m, kw, threads, ran=True):
        O.FFT_WORKERS = threads
        O.fft3(np.zeros((32, 32, 32)))
        t0 = time.perf_counter()
        out = O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos if ran else None, None, **kw)
        dt = time.perf_counter() - t0
        print(json.dumps({"cpu_full": name, "cores": threads, "seconds": round(dt, 2), "n_iter": out["n_iter"],
                          "last_rel": out["rel"][-1] if out["rel"] else None}), flush=True)

    m1 = mocks.small_periodic()
    for threads in (cores, 1):
        for start in (O.START_PLAIN, O.START_FFTA):
            run(f"64^3 periodic, 6 updates, start {start}", m1, dict(start=start, tol=0.0, max_iter=6), threads)
    m2 = mocks.survey_shell_512()
    for threads in (cores, 1):
        run("512^3 survey shell to 1e-6, Eq. approx2 start", m2, dict(start=O.START_FFTA, tol=1e-6, max_iter=80),
            threads)
    del m2
    mem_gb = 0.0
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                mem_gb = int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    if not args.cpu_full_1024:
        return
    if mem_gb >= 180:
        m5 = mocks.large_periodic_1024(los_mode=0, device="cpu")
        run("1024^3 periodic radial, 6 updates", m5, dict(start=O.START_FFTA, tol=0.0, max_iter=6), cores, ran=False)
    else:
        print(json.dumps({"cpu_full": "1024^3 periodic", "skipped": f"{mem_gb:.0f} GB host memory available"}))


def cpu_sample_text(n_iter, stages, cores, cpu_s):
    return (f"FP64 oracle on the full 512^3 workload, stage by stage: mesh stages at full size "
            f"(smoothing, delta, line of sight, start, one update x {n_iter} updates), deposit and "
            f"shift of all galaxies and {RAN_SAMPLE} of the randoms scaled to all; FFT on {cores} "
            f"threads; stage seconds {json.dumps(stages)}; {cpu_s:.1f} s of CPU work")


def kernel_sources_sha1():
    import glob
    import hashlib
    d = os.path.join(ROOT, "paper_1504_02591_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(d, "*.cu")) + glob.glob(os.path.join(d, "*.cuh")) +
                   glob.glob(os.path.join(d, "*.h")))
    h = hashlib.sha1()
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu capture, if the kernels have not changed since."""
    path = os.path.join(ROOT, "profiles", "traffic_shell512.txt")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("sources_sha1") != kernel_sources_sha1():
        return None
    return rec.get("kernels", {}).get(kernel)


def reference_arm(args):
    """The oracle as the reference arm: one warm-up per step on a small mesh, the once-per-reconstruction
    stages timed once at full size, then each timed step one full-size update of Eq. iterative."""
    import numpy as np
    from oracle import recon_oracle as O
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    n_iter = 13                                   # updates of the GPU arm's Eq. approx2 start
    m = workload(args.mesh)
    for _ in range(args.warmup):                  # warm the FFT plans and thread pool (64^3 update)
        d = np.random.default_rng(0).standard_normal((64, 64, 64))
        rh = O.rhat_field(64, 500.0, (0.0, 250.0, 250.0), O.LOS_RADIAL)
        O.update(O.start_estimate(d, 2.0, 0.7, 500.0, rh)[0], d, 2.0, 0.7, 500.0, rh)
    _, stages, _ = oracle_stages(m, 1, cores)
    p = m.params()
    n, L = p["n"], p["L"]
    # one update at full size per timed step, on the same delta and start
    rho_g_s = O.smooth(O.cic_deposit(m.galaxies.pos, None, n, L), p["R"], L)
    rho_r = O.cic_deposit(m.randoms.pos[:RAN_SAMPLE], None, n, L)
    scale_r = len(m.randoms.pos) / RAN_SAMPLE
    delta, _, _, _ = O.overdensity_randoms(rho_g_s, O.smooth(rho_r, p["R"], L) * scale_r,
                                           float(len(m.galaxies.pos)), float(len(m.randoms.pos)),
                                           p["mask_frac"], int(np.count_nonzero(rho_r > 0)))
    del rho_g_s, rho_r
    rhat = O.rhat_field(n, L, p["observer"], p["los_mode"])
    psi, _ = O.start_estimate(delta, p["b"], p["f"], L, rhat, O.START_FFTA)
    upd = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        psi = O.update(psi, delta, p["b"], p["f"], L, rhat)
        upd.append(time.perf_counter() - t0)
    stages["update"] = round(statistics.mean(upd), 3)
    value = (sum(v for k, v in stages.items() if k != "update") + n_iter * stages["update"]) * 1000.0
    step_ms = statistics.mean(upd) * 1000.0
    sample = (f"each timed step one full-size (512^3) update of Eq. iterative by the FP64 oracle; the "
              f"once-per-reconstruction stages timed once at full size (deposit and shift on all galaxies "
              f"and {RAN_SAMPLE} randoms, scaled to all); value = stages + {n_iter} updates; FFT on "
              f"{cores} threads; stage seconds {json.dumps(stages)}")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.mesh), "parallelism": "replicas"},
            "cpu_baseline": {"value": round(value, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cufft_context(n, steps=10):
    """cuFFT (through torch.fft) on the same 512^3 r2c / c2r shapes, timed with CUDA events: context
    only, never on the library's path.  One update of the iteration applies 3 c2r and 3 r2c."""
    import torch
    x = torch.randn((n, n, n), device="cuda", dtype=torch.float32)
    X = torch.fft.rfftn(x)
    y = torch.fft.irfftn(X, s=(n, n, n))
    torch.cuda.synchronize()

    def t(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    r2c = t(lambda: torch.fft.rfftn(x, out=X))
    c2r = t(lambda: torch.fft.irfftn(X, s=(n, n, n), out=y))
    del x, X, y
    torch.cuda.empty_cache()
    return {"r2c_ms": round(r2c, 4), "c2r_ms": round(c2r, 4), "update_transforms_ms": round(3 * (r2c + c2r), 4),
            "note": f"cuFFT via torch.fft on {n}^3 float32, out of place, context only (not on the library path)"}


def large_periodic(args, timed, peak):
    """The large periodic run: 1024^3 mesh, 1e8 particles, b = 1, f = 0.74, R = 10, uniform mean
    density, 6 updates from the Eq. approx2 start, shift of every particle; fixed and radial line of
    sight, and radial with the lognormal transform.  A step is deposit -> smooth -> 6 updates ->
    shift; the update's HBM fraction comes from the per-kernel CUDA events of one extra step."""
    import torch
    from paper_1504_02591_gb300 import binding, mocks
    m = mocks.large_periodic_1024(los_mode=0)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    sg = torch.empty((len(gal), 3), dtype=torch.float32, device="cuda")
    out = {"workload": "periodic 1024^3, L=2500 Mpc/h, 1e8 Zel'dovich particles (464^3 lattice + jitter), "
                       "uniform mean density, b=1 f=0.74 R=10, 6 updates from the Eq. approx2 start",
           "n_particles": len(gal)}
    variants = [("fixed", dict(los_mode=1, observer=(1.0, 0.0, 0.0))), ("radial", {}),
                ("radial_lognormal", dict(lognormal=True))]
    k = max(1, min(3, args.steps))
    for name, over in variants:
        r = binding.Recon.from_mock(m, **over)

        def step():
            r.deposit(gal, None, None, None)
            r.smooth()
            r.iterate(binding.START_FFTA, 0.0, 6)
            r.shift(gal, True, out=sg)

        step()
        ms = timed(k, step) / k
        res = {"ms": round(ms, 3)}
        if name == "radial":
            r.reset_timing()
            r.set_timing(True)
            step()
            r.set_timing(False)
            kt = r.timing()
            # one update = one launch of each of its four passes (per-launch means over the step)
            upd = [kk for kk in ("k_iter", "line_inv", "z_proj", "line_fwd") if kt[kk][0] > 0]
            upd_ms = sum(kt[kk][1] / kt[kk][0] for kk in upd)
            upd_bytes = sum(kt[kk][2] / kt[kk][0] for kk in upd)
            res["update_ms"] = round(upd_ms, 4)
            res["update_hbm_frac"] = round(upd_bytes / (upd_ms * 1e-3) / 1e9 / peak, 4)
            res["kernels"] = {kk: {"launches": v[0], "ms": round(v[1], 3),
                                   "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] > 0 else None}
                              for kk, v in kt.items() if v[0] > 0}
        out[name] = res
        r.close()
    del gal, sg
    torch.cuda.empty_cache()
    return out


def small_periodic_box(args, timed):
    """The small plain-method case: 64^3 periodic box (L = 1000, 2e5 galaxies, 2e6 randoms, b = 2,
    f = 0.74, R = 15, observer 1500 Mpc/h off the centre), 6 updates from each start; a step is
    deposit -> smooth -> 6 updates -> shift of galaxies and randoms (device-resident)."""
    import torch
    from paper_1504_02591_gb300 import binding, mocks
    m = mocks.small_periodic()
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    r = binding.Recon.from_mock(m)
    sg = torch.empty((len(gal), 3), dtype=torch.float32, device="cuda")
    sr = torch.empty((len(ran), 3), dtype=torch.float32, device="cuda")
    out = {"workload": "periodic 64^3, L=1000 Mpc/h, 2e5 galaxies + 2e6 randoms, b=2 f=0.74 R=15, 6 updates"}
    for name, start in (("uncorrected", binding.START_PLAIN), ("eq_approx2", binding.START_FFTA)):
        def step():
            r.deposit(gal, None, ran, None)
            r.smooth()
            r.iterate(start, 0.0, 6)
            r.shift(gal, True, out=sg)
            r.shift(ran, False, out=sr)
        for _ in range(3):
            step()
        k = max(5, args.steps)
        out[name] = {"ms": round(timed(k, step) / k, 4)}
    r.close()
    return out


def paper_diagnostics(m_bench, r_main):
    """Sec. 5.2 (Tables 2-3) on the benchmark survey: the mean radial ratio (Eq. ratio) of the
    real-space galaxies' displacement Z[delta_real/b] to the n-th iterate, at every galaxy, outliers
    (above 3 or below -1) cut, for n = 0..7 from the uncorrected and the Eq. approx2 starts, and the
    iteration from which the mean changes by at most 0.01 (the rule of Sec. 5.2); plus the Sec. 4.1
    Helmholtz split of the converged displacement along x (irrotational / solenoidal ratio).  All on
    the GPU (recon_radial_ratio, recon_helmholtz_x, recon_ratio_stats)."""
    import torch
    from paper_1504_02591_gb300 import binding, mocks
    out = {}
    # the benchmark survey, and the same survey geometry with a spectrum turned over at
    # k = 0.02 h/Mpc (bounded bulk flows), where the paper's Tables 2-3 pattern converges to 1
    for label, m in (("benchmark_survey", m_bench),
                     ("turnover_survey", mocks.survey_shell_512(seed=40, k_turn=0.02))):
        out[label] = radial_ratio_table(m)
    # Sec. 4.1 on a plane-parallel periodic box: the Helmholtz split of the reconstructed
    # displacement along the fixed line of sight x (the paper's Fig. 2 statistic)
    mp = mocks.periodic_box(3500.0, 512, 4_000_000, 0, 1.85, 0.74, 10.0, (1.0, 0.0, 0.0), 41, 42, 43,
                            los_mode=1, uniform=True)
    r = binding.Recon.from_mock(mp)
    r.deposit(torch.from_numpy(mp.galaxies.pos).cuda(), None, None, None)
    r.smooth()
    r.iterate(binding.START_FFTA, 1e-6, 80)
    psi = r.get_psi()
    ga, cb = r.helmholtz_x(psi[0])
    out["helmholtz_x_plane_parallel"] = {
        ax: {"all": [round(v, 4) for v in r.ratio_stats(ga[j], cb[j], -1e300, 1e300)[:2]],
             "cut_-1_3": [round(v, 4) for v in r.ratio_stats(ga[j], cb[j])[:3]]} for j, ax in enumerate("xyz")}
    r.close()
    out["note"] = ("radial ratio at every galaxy, Psi_real from the same galaxies before their redshift-space "
                   "shift; paper (mock, Table 3): uncorrected start 0.80 -> 1.10 -> 0.96 ..., converges after 6; "
                   "Eq. approx2 start 1.04, after 2 (its solve uses f where this build uses beta = f/b); "
                   "Helmholtz x ratio (Fig. 2, N-body Psi_true, R=10): mean 0.75, sigma 2.50")
    del psi, ga, cb
    torch.cuda.empty_cache()
    return out


def radial_ratio_table(m):
    """Mean radial ratio (Psi_real . r)/(Psi_n . r) over the galaxies for n = 0..7 from both starts,
    and the iteration after which the mean changes by at most 0.01 (the rule of Sec. 5.2, as the
    oracle's converged_at reads it); plus the FD method's ratio."""
    import torch
    from paper_1504_02591_gb300 import binding, diagnostics
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    p = m.params()

    def psi_of(pos, f, start, n_it):
        r = binding.Recon.from_mock(m, f=f)
        r.deposit(pos, None, ran, None)
        r.smooth()
        r.iterate(start, 0.0, n_it)
        out = r.get_psi()
        r.close()
        return out

    real = psi_of(torch.from_numpy(m.galaxies_real.pos).cuda(), 0.0, binding.START_PLAIN, 1)
    psi_s = psi_of(gal, 0.0, binding.START_PLAIN, 1)           # Z[delta/b] of the redshift-space data
    out = {}
    r = binding.Recon.from_mock(m)
    r.deposit(gal, None, ran, None)
    r.smooth()
    for name, start in (("uncorrected", binding.START_PLAIN), ("eq_approx2", binding.START_FFTA)):
        c = binding.start_coefficient(start, p["f"] / p["b"])
        rows = [r.radial_ratio(real, (1.0 - c) * psi_s, gal)[:3]]
        for n in range(1, 8):
            r.iterate(start, 0.0, n)
            rows.append(r.radial_ratio(real, r.get_psi(), gal)[:3])
        means = [x[0] for x in rows]
        out[name] = {"mean_sigma_cut": [[round(v, 4) for v in x] for x in rows],
                     "converged_at": diagnostics.converged_at(means)}
    # the finite-difference method of Sec. 2.1 on the same redshift-space delta (Table 1's FD row)
    r.deposit(gal, None, ran, None)
    r.smooth()
    t0 = time.perf_counter()
    psi_fd, it, res, st = r.fd_solve(1e-6, 300)
    fd_s = time.perf_counter() - t0
    out["finite_difference"] = {"mean_sigma_cut": [round(v, 4) for v in r.radial_ratio(real, psi_fd, gal)[:3]],
                                "bicgstab_iterations": it, "residual": res, "seconds": round(fd_s, 3)}
    r.close()
    del gal, ran, real, psi_s, psi_fd
    torch.cuda.empty_cache()
    return out


def batch_bench(args):
    """The batched workload: 64 mocks (N from {256, 384, 512}, 2e5-1e6 galaxies, 30-50x randoms,
    per-mock b and f, shell surveys and periodic boxes) reconstructed to 1e-6 from the Eq. approx2
    start in one recon_batch_run call (a CUDA graph per mock, launched back to back).  The first
    call tunes each size class (not timed); each timed call is the whole batch, from the call to
    its return."""
    import torch
    from paper_1504_02591_gb300 import binding, mocks
    work = mocks.batch_workload_device(64, 100)
    sizes = [w["params"]["n"] for w in work]
    particles = sum(len(w["gal"]) + (len(w["ran"]) if w["ran"] is not None else 0) for w in work)
    st, res = binding.batch_run(work, start=binding.START_FFTA, tol=args.tol, max_iter=args.max_iter)  # tunes
    outs = [(r["shift_gal"], r["shift_ran"]) for r in res]   # shift buffers allocated once, as in the step
    k = max(1, min(2, args.steps))
    times = []
    for _ in range(k):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, res = binding.batch_run(work, start=binding.START_FFTA, tol=args.tol, max_iter=args.max_iter, out=outs)
        times.append(time.perf_counter() - t0)
    wall = statistics.mean(times)
    item_ms = [r["ms"] for r in res]
    by_n = {}
    for n, r in zip(sizes, res):
        d = by_n.setdefault(str(n), {"mocks": 0, "ms": [], "n_iter": []})
        d["mocks"] += 1
        d["ms"].append(r["ms"])
        d["n_iter"].append(r["n_iter"])
    out = {"workload": "64 mocks, N in {256, 384, 512}, 2e5-1e6 galaxies, randoms 30-50x, b in [1.5, 2.5], "
                       "f in [0.6, 0.8], shell surveys and periodic boxes, converged to 1e-6",
           "status": int(st), "ok": sum(1 for r in res if r["status"] == binding.OK),
           "particles": int(particles), "wall_s": round(wall, 4), "mocks_per_s": round(len(work) / wall, 3),
           "ms_per_mock": round(1000.0 * wall / len(work), 3),
           "item_ms_sum": round(sum(item_ms), 2),
           "classes": {n: {"mocks": d["mocks"], "mean_ms": round(statistics.mean(d["ms"]), 3),
                           "mean_updates": round(statistics.mean(d["n_iter"]), 2)} for n, d in sorted(by_n.items())},
           "plans": {str(n): binding.batch_plan(n) for n in (256, 384, 512)},
           "launch": "one CUDA graph per mock (conditional WHILE loop), launched back to back, smallest mesh "
                     "first; the host builds each graph while the device runs the ones before it"}
    del work, res, outs
    torch.cuda.empty_cache()
    return out


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1504_02591_gb300 import binding, warmstart

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    m = workload(args.mesh)
    gal = torch.from_numpy(m.galaxies.pos).cuda()
    ran = torch.from_numpy(m.randoms.pos).cuda()
    r = binding.Recon.from_mock(m)
    if args.host_loop:
        r.set_option(binding.OPT_GRAPH, 0)
    if args.particle_order == "retained":
        r.set_option(binding.OPT_DEPOSIT_PATH, binding.PATH_SORTED)
        r.set_option(binding.OPT_REUSE_SORT, 1)
    if args.plane_batch is not None:
        r.set_option(binding.OPT_PLANE_BATCH, args.plane_batch)
    sg = torch.empty((len(gal), 3), dtype=torch.float32, device="cuda")
    sr = torch.empty((len(ran), 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    info = {}

    def step(start=binding.START_FFTA):
        r.deposit(gal, None, ran, None)
        r.smooth()
        n_it, rel, st = r.iterate(start, args.tol, args.max_iter)
        r.shift(gal, True, out=sg)
        r.shift(ran, False, out=sr)
        info["n_iter"], info["rel"], info["status"] = n_it, rel, st

    def barrier():
        if ws > 1:
            dist.barrier()

    def timed(k, fn):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), "cuda")

    # the learned warm start: the network trained for this workload on other seeds
    # (train_warmstart.py), run on the mesh coarsened `level` times, then the same iteration from its
    # prediction to the same stopping rule.  It is the timed path when its weights are present.
    net, level = None, 0
    wpath = warmstart.default_weights_path()
    if not args.no_warm and os.path.exists(wpath):
        net, level = warmstart.load(wpath)

    def step_warm(gal_in=gal, ran_in=ran, sg_out=sg, sr_out=sr):
        r.deposit(gal_in, None, ran_in, None)
        r.smooth()
        feat = r.start_features(binding.START_FFTA, level)
        info["warm_feat"] = feat
        y = net.forward(feat)
        n_it, rel_w, st = r.iterate_from(y, args.tol, args.max_iter, level)
        r.shift(gal_in, True, out=sg_out)
        r.shift(ran_in, False, out=sr_out)
        info["n_iter"], info["rel"], info["status"] = n_it, rel_w, st

    main_step = step_warm if net is not None else step
    for _ in range(max(3, args.warmup)):
        main_step()
    # timed region: the library's default path (iteration as one CUDA graph), no per-kernel events
    r.reset_timing()
    l0 = net.launch_count() if net is not None else 0
    clocks = Clocks(local)
    clocks.start()
    total_ms = timed(args.steps, main_step)
    clk = clocks.stop()
    launches = sum(v[0] for v in r.timing().values()) + ((net.launch_count() - l0) if net is not None else 0)
    n_iter, rel = info["n_iter"], info["rel"]
    ms_per_step = total_ms / args.steps
    warm = None
    if net is not None:
        feat = info.pop("warm_feat")
        net_ms = timed(3, lambda: net.forward(feat)) / 3
        warm = {"ms": round(ms_per_step, 4), "n_iter": n_iter, "final_rel": rel, "network_ms": round(net_ms, 4),
                "level": level, "grid": args.mesh >> level, "c1": net.c1,
                "weights": os.path.relpath(wpath, os.path.dirname(os.path.abspath(__file__)))}
    # the plain iteration from the Eq. approx2 start on the same input
    for _ in range(2):
        step()
    plain_ms = timed(args.steps, step) / args.steps
    plain = {"ms": round(plain_ms, 4), "n_iter": info["n_iter"], "final_rel": info["rel"], "start": "Eq. approx2"}
    info_plain_iter = info["n_iter"]
    # per-kernel CUDA-event timings over the same number of steps (events around every launch on
    # the library's stream; the iteration runs host-driven so that each launch can be bracketed)
    r.reset_timing()
    r.set_timing(True)
    timed(args.steps, main_step)
    r.set_timing(False)
    kt = r.timing()

    # the uncorrected start (c = 0) on the same input
    unc_steps = 2
    unc_ms = timed(unc_steps, lambda: step(binding.START_PLAIN)) / unc_steps
    unc_iter = info["n_iter"]

    # roofline of the dominant kernel (largest share of device time in the timed region)
    peak, peak_kind = peaks()
    busy = {k: v for k, v in kt.items() if v[0] > 0 and v[1] > 0}
    dom = max(busy, key=lambda k: busy[k][1])
    cnt, ms_k, by = busy[dom]
    achieved = (by / cnt) / (ms_k / cnt * 1e-3) / 1e9
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / sum(x[1] for x in busy.values()), 4),
                   "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] > 0 else None}
               for k, v in busy.items()}
    if warm:
        kernels["unet_forward"] = {"launches": args.steps, "ms": round(warm["network_ms"] * args.steps, 3),
                                   "share": None, "GBps": None}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        gal_h = torch.from_numpy(m.galaxies.pos).pin_memory()
        ran_h = torch.from_numpy(m.randoms.pos).pin_memory()
        sg_h = torch.empty((len(gal_h), 3), dtype=torch.float32).pin_memory()
        sr_h = torch.empty((len(ran_h), 3), dtype=torch.float32).pin_memory()

        def step_e2e():
            if net is not None:
                step_warm(gal_h, ran_h, sg_h, sr_h)
                return
            r.deposit(gal_h, None, ran_h, None)
            r.smooth()
            r.iterate(binding.START_FFTA, args.tol, args.max_iter)
            r.shift(gal_h, True, out=sg_h)
            r.shift(ran_h, False, out=sr_h)

        step_e2e()
        k_e = max(1, min(args.steps, 3))
        e_ms = timed(k_e, step_e2e) / k_e
        npart = len(gal_h) + len(ran_h)
        # positions read over the link: every tracer by the deposit, then by its shift, except the
        # randoms in the retained order (their shift reuses the deposit's sorted records)
        reread = len(gal_h) if args.particle_order == "retained" else npart
        e2e = {"value": round(job_value(e_ms, ws), 4), "unit": "ms", "h2d_bytes_per_step": int((npart + reread) * 24),
               "d2h_bytes_per_step": int(npart * 12), "ms_per_step": round(e_ms, 4)}

    small = small_periodic_box(args, timed)
    diag = paper_diagnostics(m, r) if not args.no_diag else None
    cufft = cufft_context(args.mesh) if not args.no_cufft else None
    batch = batch_bench(args) if not args.no_batch else None
    large = large_periodic(args, timed, peak) if not args.no_large else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        v, stages, cpu_s = oracle_stages(m, info_plain_iter, cores)
        cpu = {"value": round(v, 1), "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": cpu_sample_text(info_plain_iter, stages, cores, cpu_s)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(job_value(ms_per_step, ws), 4), "unit": "ms", "n_gpus": ws,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args.mesh), "mesh": args.mesh, "box": 3500.0,
                       "n_gal": len(gal), "n_ran": len(ran), "n_iter": n_iter, "final_rel": rel,
                       "start": "learned warm start (U-Net on the 4x coarsened mesh)" if warm else "Eq. approx2",
                       "l2": "inputs larger than L2 (each field 539 MB), no flush",
                       "parallelism": "replicas" if ws > 1 else "single",
                       "iteration_loop": "host" if args.host_loop else "cuda graph",
                       "particle_order": args.particle_order},
            "path": "learned warm start" if warm else "Eq. approx2 start",
            "warm_start": warm,
            "plain": plain,
            "uncorrected_start": {"ms": round(unc_ms, 4), "n_iter": unc_iter},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                         "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": recorded_traffic(dom), "alg_bytes_per_launch": by / cnt,
                         "ms_per_launch": round(ms_k / cnt, 5)},
            "kernels": kernels,
            "small_periodic_64": small,
            "paper_diagnostics": diag,
            "large_periodic_1024": large,
            "batch": batch,
            "cufft_context": cufft,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if net is not None:
        net.close()
    r.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.cpu_full:
        cpu_full(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
