"""Host-side checks of the C-ABI library: it builds, loads without a GPU, exports every symbol that
include/recon.h declares, and validates parameters (no device work is launched here)."""
import ctypes as C
import os
import re

import pytest

from paper_1504_02591_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_02591_gb300 import _build
    path = _build.build()
    return C.CDLL(path)


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(recon_\w+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(binding.ABI_SYMBOLS)


def declared_constants():
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\bRECON_([A-Z0-9_]+)\s*=\s*(-?\d+)", src)}


def test_header_constants_and_binding_agree():
    consts = declared_constants()
    assert len(consts) > 40
    kinds = [k.replace("_", "") for k in binding.KERNEL_KINDS]
    for name, value in consts.items():
        if name == "K_COUNT":
            assert value == len(binding.KERNEL_KINDS)
        elif name.startswith("K_"):
            assert kinds.index(name[2:].replace("_", "").lower()) == value, name
        else:
            assert getattr(binding, name) == value, name


def test_batch_flags_are_validated(lib):
    lib.recon_batch_run.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
    for bad in (4, 8, -1):   # rejected before any device work
        assert lib.recon_batch_run(None, 0, None, bad) == binding.ERR_INVALID_ARG
    assert lib.recon_batch_run(None, -1, None, 0) == binding.ERR_INVALID_ARG


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_workspace_bytes_and_validation(lib):
    binding._lib = None
    binding.load()
    for n in (32, 48, 64, 96, 128, 256, 384, 512, 1024):
        p = binding.make_params(n, 1000.0, 2.0, 0.7, 10.0, (0, 0, 0))
        ws = binding.workspace_bytes(p)
        assert ws >= 5 * 4 * n ** 3
    for bad in (dict(n=100), dict(n=16), dict(b=0.0), dict(L=-1.0), dict(R=-1.0)):
        kw = dict(n=64, L=1000.0, b=2.0, f=0.7, R=10.0, observer=(0, 0, 0))
        kw.update(bad)
        with pytest.raises(binding.ReconError) as e:
            binding.workspace_bytes(binding.make_params(**kw))
        assert e.value.status == binding.ERR_INVALID_ARG
    p = binding.make_params(64, 1000.0, 2.0, 0.7, 10.0, (0, 0, 0), los_mode=binding.LOS_FIXED)
    with pytest.raises(binding.ReconError):
        binding.workspace_bytes(p)       # a fixed LOS needs a non-zero direction
    p = binding.make_params(64, 1000.0, 2.0, 0.7, 10.0, (1, 0, 0))
    p.nmesh[2] = 32
    with pytest.raises(binding.ReconError):
        binding.workspace_bytes(p)       # non-cubic meshes are rejected


def test_status_strings(lib):
    lib.recon_status_str.restype = C.c_char_p
    for s in range(9):
        assert lib.recon_status_str(s)
    lib.recon_destroy.argtypes = [C.c_void_p]
    assert lib.recon_destroy(None) == 0


def test_start_coefficient_matches_the_oracle(lib):
    """recon_start_coefficient (host only) gives the c of Sec. 5.2's starts as the oracle does."""
    from oracle import recon_oracle as O
    binding._lib = None
    binding.load()
    for start in (binding.START_PLAIN, binding.START_APPROX1, binding.START_FFTA):
        for beta in (0.0, 0.2, 0.4, 0.74, 3.0):
            assert binding.start_coefficient(start, beta) == pytest.approx(O.start_coefficient(start, beta), rel=1e-15)
    for start, beta in ((3, 0.4), (-1, 0.4), (0, -0.1), (2, float("nan"))):
        with pytest.raises(binding.ReconError) as e:
            binding.start_coefficient(start, beta)
        assert e.value.status == binding.ERR_INVALID_ARG


def test_diagnostic_convergence_rule_matches_the_oracle():
    """The package's host rule for the paper's convergence iteration (Sec. 5.2) agrees with the
    oracle's, which the paper's own Tables 2 and 3 pin (tests/golden/iteration_tables.txt)."""
    import numpy as np
    from oracle import recon_oracle as O
    from paper_1504_02591_gb300 import diagnostics
    rows = [ln.split() for ln in open(os.path.join(ROOT, "tests", "golden", "iteration_tables.txt"))
            if ln.strip() and not ln.startswith("#") and not ln.startswith("converged")]
    seqs = {}
    for t, s, n, m, *_ in rows:
        seqs.setdefault((t, s), []).append((int(n), float(m)))
    for seq in seqs.values():
        means = [m for _, m in sorted(seq)]
        assert diagnostics.converged_at(means) == O.converged_at(means)
    rng = np.random.default_rng(3)
    for _ in range(500):
        means = list(1.0 + np.cumsum(rng.choice([-1, 1], 8) * rng.choice([0.0, 0.005, 0.01, 0.02, 0.1], 8)))
        assert diagnostics.converged_at(means) == O.converged_at(means)
    assert diagnostics.converged_at([0.9]) == 0


def test_no_cpu_fallback(tmp_path):
    """The product path has no CPU fallback: a missing library and a missing GPU both fail loudly."""
    saved = binding._lib
    try:
        binding._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            binding.load(str(tmp_path / "librecon_gb300.so"))
    finally:
        binding._lib = saved
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="only on the GPU"):
        binding.Recon(64, 1000.0, 2.0, 0.7, 10.0, (0.0, 0.0, 0.0))
