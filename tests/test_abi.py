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
    lib.mlpg_step_batch.restype = ctypes.c_int
    assert lib.mlpg_step_batch(None, None, 1, None) == -1
    st = (ctypes.c_int * 1)(12345)
    assert lib.mlpg_step_batch((ctypes.c_void_p * 1)(None), (ctypes.c_double * 1)(0.1), 1, st) == -1
    assert st[0] == 12345          # argument errors leave the per-context statuses unwritten
    lib.mlpg_last_error.restype = ctypes.c_char_p
    assert lib.mlpg_last_error(None) == b"null context"


def test_product_never_imports_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2008_02205_gb300")
    for dp, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.lower() or f.endswith(".py") and "import oracle" not in txt, f


def _c_layout(tmp_path, struct, fields):
    """Offsets and size of a header struct, as gcc lays it out on this machine."""
    src = tmp_path / f"{struct}.c"
    body = "".join(f'    printf("{f} %zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "mlpg.h"\nint main(void) {\n'
                   f'{body}    printf("__size__ %zu\\n", sizeof({struct}));\n    return 0;\n}}\n')
    exe = tmp_path / struct
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("struct,cls", [("mlpg_options", "Options"), ("mlpg_stats", "Stats")])
def test_binding_structs_match_header_layout(tmp_path, struct, cls):
    import paper_2008_02205_gb300 as pkg
    C = getattr(pkg, cls)
    names = [f for f, _ in C._fields_]
    want = _c_layout(tmp_path, struct, names)
    for f in names:
        assert getattr(C, f).offset == want[f], (struct, f)
    assert ctypes.sizeof(C) == want["__size__"]


def test_default_options(lib):
    import paper_2008_02205_gb300 as pkg
    o = pkg.mlpg_default_options()
    assert (o.precision, o.inner_restart, o.mixed_restart, o.check_every) == (0, 20, 20, 3)
    assert (o.mixed_reorth, o.mixed_half_prec, o.rk_order) == (0, 1, 1)
    assert (o.inner_tol, o.outer_tol, o.mixed_inner_tol) == (1e-12, 1e-12, 1e-2)


@pytest.mark.parametrize("bad", ["points_dim", "omega_cols", "extent", "weights", "sigma_t", "sigma_s", "q"])
def test_binding_rejects_mismatched_arrays_before_the_library_reads_them(lib, bad):
    # the C side reads n * dim, n, 3 m and m values from the pointers it is given:
    # the binding checks every shape first (no device needed, nothing reaches C)
    import numpy as np
    import paper_2008_02205_gb300 as pkg
    n, m = 16, 4
    args = dict(points=np.zeros((n, 2)), kernel_extent=np.ones(n), omega=np.tile([1.0, 0, 0], (m, 1)),
                w=np.ones(m), sigma_t=np.ones(n), sigma_s=np.zeros(n), q=np.ones(n))
    short = {"points_dim": ("points", np.zeros((n, 3))), "omega_cols": ("omega", np.zeros((m, 2))),
             "extent": ("kernel_extent", np.ones(n - 1)), "weights": ("w", np.ones(m + 1)),
             "sigma_t": ("sigma_t", np.ones(n - 1)), "sigma_s": ("sigma_s", np.ones((n, 1))),
             "q": ("q", np.ones(2 * n))}[bad]
    args[short[0]] = short[1]
    with pytest.raises(ValueError):
        pkg.mlpg_create(pkg.mlpg_default_options(dim=2), **args)


@pytest.mark.parametrize("field,value", [("dim", 4), ("dim", 1), ("rk_order", 3), ("rk_order", -1),
                                         ("mixed_reorth", 2), ("mixed_half_prec", 2), ("outer_method", 2),
                                         ("inner_restart", 0), ("inner_restart", 33), ("outer_restart", 33),
                                         ("mixed_restart", 0), ("check_every", 0), ("c", 0.0), ("c", -1.0),
                                         ("tau_factor", -0.5), ("precision", 5)])
def test_invalid_options_are_rejected_before_any_device_call(lib, field, value):
    # option and size checks run before the library touches CUDA: *out stays NULL
    import numpy as np
    import paper_2008_02205_gb300 as pkg
    o = pkg.mlpg_default_options()
    setattr(o, field, value)
    n, m = 16, 4
    arr = [np.zeros((n, 2)), np.ones(n), np.tile([1.0, 0.0, 0.0], (m, 1)), np.ones(m), np.ones(n), np.zeros(n),
           np.ones(n)]
    ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arr]
    out = ctypes.c_void_p()
    L = pkg.load_library()
    st = L.mlpg_create(ctypes.byref(o), n, ptrs[0], ptrs[1], m, ptrs[2], ptrs[3], ptrs[4], ptrs[5], ptrs[6],
                       ctypes.byref(out))
    assert st == pkg.MLPG_ERR_ARG and not out.value


def test_empty_box_and_tiny_problems_are_rejected(lib):
    import numpy as np
    import paper_2008_02205_gb300 as pkg
    L = pkg.load_library()
    for n, lohi in ((16, ((0.0, 0.0), (1.0, 0.0))), (3, ((0.0, 0.0), (1.0, 1.0)))):
        o = pkg.mlpg_default_options(lo=lohi[0], hi=lohi[1])
        arr = [np.zeros((n, 2)), np.ones(n), np.array([[1.0, 0.0, 0.0]]), np.ones(1), np.ones(n), np.zeros(n),
               np.ones(n)]
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arr]
        out = ctypes.c_void_p()
        st = L.mlpg_create(ctypes.byref(o), n, ptrs[0], ptrs[1], 1, ptrs[2], ptrs[3], ptrs[4], ptrs[5], ptrs[6],
                           ctypes.byref(out))
        assert st == pkg.MLPG_ERR_ARG and not out.value


def test_binding_status_codes_match_the_header():
    import paper_2008_02205_gb300 as pkg
    txt = open(HEADER).read()
    for name, val in re.findall(r"\b(MLPG_(?:OK|ERR_[A-Z_]+))\s*=\s*(-?\d+)", txt):
        assert getattr(pkg, name) == int(val), name
        assert pkg.STATUS[int(val)] == name
