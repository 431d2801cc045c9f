"""The C-ABI library loads and exports every entry point declared in
include/mlpg.h (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlpg.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mlpg_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_02205_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_calls():
    names = _declared()
    for must in ("mlpg_create", "mlpg_integrate", "mlpg_assemble", "mlpg_step", "mlpg_scalar_flux"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_entry_point():
    import paper_2008_02205_gb300 as pkg
    for n in _declared():
        assert hasattr(pkg, n), n


def test_null_arguments_rejected_without_device(lib):
    # argument checks happen before any CUDA call
    lib.mlpg_create.restype = ctypes.c_int
    assert lib.mlpg_create(None, 0, None, None, 0, None, None, None, None, None, None) == -1
    lib.mlpg_last_error.restype = ctypes.c_char_p
    assert lib.mlpg_last_error(None) == b"null context"


def test_product_never_imports_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2008_02205_gb300")
    for dp, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.lower() or f.endswith(".py") and "import oracle" not in txt, f
