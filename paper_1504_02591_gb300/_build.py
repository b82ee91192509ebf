"""Build the C-ABI shared library (librecon_gb300.so) in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel; a unit is rebuilt only when a source or header it may
include is newer than its object file, or the flags changed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "librecon_gb300.so")

SOURCES = ["recon.cu", "cic.cu", "conv.cu", "bricks.cu", "loop.cu", "batch.cu", "diag.cu", "fd.cu", "unet.cu", "unet_tc.cu", "warm.cu", "inst_a.cu", "inst_b.cu", "inst_c.cu", "inst_d.cu", "inst_e.cu", "inst_f.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-O2",
         "-I" + os.path.join(ROOT, "include")] + ARCH


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librecon_gb300.so")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "recon.h"))
    return hs


def _flag_tag(extra):
    return hashlib.sha1(" ".join(FLAGS + list(extra)).encode()).hexdigest()[:12]


def _compile(src, extra, verbose):
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    tagf = obj + ".flags"
    tag = _flag_tag(extra)
    srcp = os.path.join(CSRC, src)
    newest = max(os.path.getmtime(p) for p in [srcp] + _headers())
    if (os.path.exists(obj) and os.path.getmtime(obj) >= newest and os.path.exists(tagf)
            and open(tagf).read() == tag):
        return obj, None
    cmd = [_nvcc(), "-c", srcp, "-o", obj] + FLAGS + list(extra)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return obj, "FAILED: " + " ".join(cmd) + "\n" + r.stdout + r.stderr
    with open(tagf, "w") as fh:
        fh.write(tag)
    return obj, (r.stdout + r.stderr) if verbose else None


def build(verbose: bool = False, extra=(), jobs: int | None = None) -> str:
    """Compile every CUDA source for sm_103a and link librecon_gb300.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, verbose), SOURCES))
    errors = [msg for _, msg in results if msg and msg.startswith("FAILED")]
    if errors:
        raise RuntimeError("\n".join(errors))
    if verbose:
        for _, msg in results:
            if msg:
                print(msg, file=sys.stderr)
    objs = [o for o, _ in results]
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [_nvcc(), "-shared", "-o", LIB] + objs + ARCH
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "-v" in sys.argv else ()))
