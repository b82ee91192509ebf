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
