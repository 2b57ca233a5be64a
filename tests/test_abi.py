"""Host-side checks of the C-ABI library: it builds, loads without a GPU and
exports every entry point include/sscg.h declares; the Python binding and the
CUDA path never reach the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_03743_gb300 import build

    return ctypes.CDLL(build.build())


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int64_t|int|const char\*|void)\s+\**\s*(sscg_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "sscg_solve" in names and "sscg_pcg_solve" in names and "sscg_mat_create_csr" in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2501_03743_gb300 import sscg

    assert set(declared_functions()) <= set(sscg.EXPORTS)


def test_status_strings_without_gpu(lib):
    lib.sscg_status_str.restype = ctypes.c_char_p
    assert lib.sscg_status_str(0) == b"converged"
    assert b"invalid" in lib.sscg_status_str(-1)


def test_storage_size_query_without_gpu(lib):
    n = ctypes.c_size_t()
    assert lib.sscg_mat_storage_bytes(ctypes.c_int64(1000), ctypes.c_int64(7000), ctypes.byref(n)) == 0
    assert n.value >= 7000 * (4 + 8 + 4 + 4) + 1001 * 4
    assert lib.sscg_mat_storage_bytes(ctypes.c_int64(0), ctypes.c_int64(0), ctypes.byref(n)) == -1


def test_no_cpu_fallback_in_product_path():
    """The package and its CUDA sources never import, load or call the oracle."""
    pkg = os.path.join(ROOT, "paper_2501_03743_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "sscg_oracle" not in text and "liboracle" not in text, f


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2501_03743_gb300 import sscg

    saved = sscg._lib
    sscg._lib = None
    try:
        with pytest.raises(ImportError):
            sscg.load(str(tmp_path / "missing.so"))
    finally:
        sscg._lib = saved


def test_newton_shifts_host_logic_matches_the_oracle():
    """The library's Newton shifts (host code, no GPU) are the oracle's: the
    Leja-ordered Chebyshev points of the interval and sigma = (hi - lo)/4."""
    import numpy as np

    import oracle
    from paper_2501_03743_gb300 import sscg

    for s, lo, hi in ((1, 0.1, 2.0), (2, 0.1, 2.0), (5, 0.05, 1.95), (8, 0.3, 7.0), (12, 1e-3, 2.0), (16, 2.0, 9.5)):
        th, sig = sscg.newton_shifts(s, lo, hi)
        tho, sigo = oracle.newton_shifts(s, lo, hi)
        assert len(th) == s - 1 and sig == sigo
        assert np.allclose(th, tho, rtol=1e-14, atol=0)
    for bad in ((0, 0.1, 2.0), (17, 0.1, 2.0), (4, 2.0, 2.0)):
        with pytest.raises(sscg.SscgError):
            sscg.newton_shifts(*bad)
