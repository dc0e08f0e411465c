"""The C-ABI library loads and exports every entry point include/gecc.h declares
(no GPU needed: only symbol lookup, no compute call)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ecc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2501_03245_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "ecc_verify_batch" in names and "ecc_fp_mul" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_2501_03245_gb300 import ecc

    for n in declared():
        assert hasattr(ecc, n), n
        assert n in ecc.exported_symbols(), n


def test_host_only_calls(lib):
    """Calls that fail argument checks before touching the GPU."""
    from paper_2501_03245_gb300 import ecc

    lib.ecc_limbs.restype = ctypes.c_int
    assert lib.ecc_limbs(0) == 8 and lib.ecc_limbs(3) == 12 and lib.ecc_limbs(4) == 8
    assert lib.ecc_limbs(7) == ecc.ECC_EINVAL
    lib.ecc_last_error.restype = ctypes.c_char_p
    assert b"unknown curve" in lib.ecc_last_error()
