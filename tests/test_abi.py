"""The C-ABI library loads and exports every function include/molt.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import pathlib
import re

from tests.conftest import ROOT


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = pathlib.Path(inc, f).read_text()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(molt_\w+)\s*\(", src, flags=re.M)
    return names


def test_header_declares_the_entry_points():
    names = declared_functions()
    for f in ("molt_create", "molt_apply_D", "molt_step", "molt_destroy", "molt_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_2007_03041_gb300 import molt as M
    if not os.path.exists(M.LIB_PATH):
        from paper_2007_03041_gb300 import build
        build.build()
    lib = ctypes.CDLL(M.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_the_header():
    from paper_2007_03041_gb300 import molt as M
    for name in declared_functions():
        if name != "molt_last_error":
            assert callable(getattr(M, name)), name


def test_binding_constants_match_the_header_enums():
    """Every enumerator `MOLT_<NAME> = <value>` of the header that the binding
    exposes as `<NAME>` carries the same value (options, kernel kinds,
    boundary types, operators, precisions, ...)."""
    from paper_2007_03041_gb300 import molt as M
    src = pathlib.Path(ROOT, "include", "molt.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    pairs = re.findall(r"\bMOLT_([A-Z0-9_]+)\s*=\s*(-?\d+)", src)
    checked = 0
    for name, value in pairs:
        if hasattr(M, name):
            assert getattr(M, name) == int(value), (name, getattr(M, name), value)
            checked += 1
    for name in ("OPT_LANES", "OPT_AXIS_STREAMS", "OPT_XLINES", "KERNEL_XLINES_ACC_SET", "KERNEL_LANES_ACC_ADD"):
        assert hasattr(M, name), name
    assert checked >= 30, checked
