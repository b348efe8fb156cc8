"""The C-ABI library loads and exports every symbol include/bsf.h declares (no GPU needed)."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bsf():
    from paper_1109_5114_gb300 import build
    build.build()
    from paper_1109_5114_gb300 import bsf as mod
    return mod


def test_every_declared_symbol_is_exported(bsf):
    names = bsf.declared_symbols()
    assert len(names) >= 14
    lib = ctypes.CDLL(bsf.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_header_constants(bsf):
    assert bsf.BSF_OK == 0 and bsf.BSF_EINVAL == -1 and bsf.BSF_EOVERFLOW == -6
    assert (bsf.BSF_ZERO, bsf.BSF_REPLICATE, bsf.BSF_SYMMETRIC) == (0, 1, 2)
    assert (bsf.BSF_FIX64, bsf.BSF_FIX128) == (1, 2)


def test_invalid_arguments_rejected_before_any_device_call(bsf):
    h = bsf.bsf_t()
    for args in [(0, 8, 4, 1, 0, -1), (8, 8, 3, 1, 0, -1), (8, 8, 4, 0, 0, -1),
                 (8, 8, 4, 4, 0, -1), (8, 8, 4, 1, 3, -1), (8, 8, 4, 1, 0, -2)]:
        assert bsf.bsf_create(ctypes.byref(h), *args) == bsf.BSF_EINVAL
    assert bsf.bsf_create(None, 8, 8, 4, 1, 0, -1) == bsf.BSF_EINVAL
    assert bsf.bsf_status(None) == bsf.BSF_EINVAL
    assert bsf.bsf_last_error(None) == b"NULL context"
    bsf.bsf_destroy(None)


def test_product_path_has_no_oracle_import():
    # the library binding and kernels never touch the oracle package
    pkg = os.path.join(ROOT, "paper_1109_5114_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_binding_refuses_to_load_without_the_library(tmp_path):
    # no fallback: a copy of the binding whose package has no built library
    # fails at import, before any call could run anywhere else
    import importlib.util
    import shutil
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_1109_5114_gb300", "bsf.py"), pkg / "bsf.py")
    spec = importlib.util.spec_from_file_location("bsf_without_library", pkg / "bsf.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError, match="not built"):
        spec.loader.exec_module(mod)
