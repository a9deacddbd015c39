"""CPU-side checks of the sm_103a library: it builds, loads, and exports every
entry point include/rbfgs.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import paper_1602_01768_gb300._binding as B
from paper_1602_01768_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:rb_status|void|const char\s*\*)\s*\**\s*(\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return names


def test_library_builds_for_sm103a():
    path = libbuild.build()
    assert os.path.exists(path)


def test_library_exports_every_declared_entry_point():
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(libbuild.build())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_entry_point_under_its_c_name():
    names = set(declared_functions())
    assert names == set(B.exported_symbols())
    for n in names:
        assert callable(getattr(B, n)), n


def test_status_strings_without_gpu():
    lib = B._lib()
    assert lib.rbfgs_status_string(B.RB_ENOTSPD).startswith(b"Cholesky")
    o = B.rbfgs_default_opts()
    assert o.q == 8 and o.prec == B.RB_FP64 and o.method == B.RB_METHOD_RBFGS
