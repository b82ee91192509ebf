#!/usr/bin/env python
"""Benchmark: milliseconds per converged 512^3 reconstruction on GB300.

One step = the whole path on one synthetic survey: CIC deposit of 6e5 galaxies and 3e7 randoms,
Gaussian smoothing and delta with the survey mask, the Fourier-space iteration from the
RSD-corrected (Eq. approx2) start until |dPsi|/|Psi| < 1e-6, and the shift of every galaxy and
random.  Inputs are resident in HBM when the timed region starts; every field (539 MB) is larger
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


CPU_MESH = 256
CPU_SCALE = (512 / CPU_MESH) ** 3 * 27.0 / (3 * 8)      # volume x log(512^3)/log(256^3)
CPU_SAMPLE = (f"oracle deposit+smooth+iterations+shift on the {CPU_MESH}^3 version of the workload "
              f"(75000 galaxies, 3750000 randoms), x{CPU_SCALE:.3f} to 512^3")


def cpu_sample(n_iter):
    """The FP64 oracle as it stands on a bounded sample of the workload, scaled to 512^3.

    Sample: the same survey shape on a 256^3 mesh with 1/8 of the tracers and the GPU's iteration
    count.  Every stage scales with the mesh volume (FFT stages as N^3 log N) or with the tracer
    count, so the time is multiplied by 8 * log(512^3)/log(256^3) = 9.
    """
    from oracle import recon_oracle as O
    from paper_1504_02591_gb300 import mocks
    m = mocks.survey_shell_512(n_gal=600_000 // 8, ran_ratio=50, n_mesh=CPU_MESH)
    t0 = time.perf_counter()
    O.reconstruct(m.params(), m.galaxies.pos, None, m.randoms.pos, None, start=O.START_FFTA,
                  tol=0.0, max_iter=n_iter)
    dt = time.perf_counter() - t0
    return dt * 1000.0 * CPU_SCALE, dt


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
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    n_iter = 13
    for _ in range(args.warmup):
        cpu_sample(n_iter)
    vals, raw = [], []
    for _ in range(args.steps):
        v, dt = cpu_sample(n_iter)
        vals.append(v)
        raw.append(dt)
    value = statistics.mean(vals)
    sample = CPU_SAMPLE + f"; {n_iter} iterations, {statistics.mean(raw):.1f} s per sample"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.mesh), "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, dt = cpu_sample(n_iter)
        cpu = {"value": round(v, 1), "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": CPU_SAMPLE + f"; {n_iter} iterations took {dt:.2f} s"}

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
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
