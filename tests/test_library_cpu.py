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
        for m in re.finditer(r"^\s*(?:rb_status|void|int|const char\s*\*)\s*\**\s*(\w+)\s*\(", text, flags=re.M):
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


def test_predicted_check_spacing_without_gpu():
    """rb_next_check_gap: half the steps a geometric fit of two checks predicts to reach tol, in [e, 8e]."""
    import math
    gap = B.rb_next_check_gap
    assert gap(32, -1, 0.0, 32, 1e-2, 1e-4) == 32          # one check only
    assert gap(32, 32, 1e-2, 64, 1e-2, 1e-4) == 256        # not falling
    assert gap(32, 32, 1e-2, 64, 2e-2, 1e-4) == 256        # rising
    assert gap(32, 32, 1e-2, 64, 5e-5, 1e-4) == 32         # already below tol
    def expect(e, k0, r0, k1, r1, tol):
        lr = math.log(r1 / r0) / (k1 - k0)
        return max(e, min(8 * e, math.floor(0.5 * math.log(tol / r1) / lr)))

    # falls by 10x per 100 steps: about 200 steps from 1e-2 to 1e-4, so the next check after about 100
    assert abs(gap(32, 0, 1e-1, 100, 1e-2, 1e-4) - 100) <= 1
    assert gap(32, 0, 1e-1, 100, 1e-2, 1e-4) == expect(32, 0, 1e-1, 100, 1e-2, 1e-4)
    # the same rate near tol: 10 predicted steps -> the minimum spacing
    r1 = 1e-4 * 10 ** 0.1
    assert gap(32, 0, r1 * 10, 100, r1, 1e-4) == 32
    # a slow fall: the cap
    assert gap(32, 0, 1.0, 100, 0.99, 1e-4) == 256
    assert gap(16, 64, 4e-3, 128, 3e-3, 1e-4) == expect(16, 64, 4e-3, 128, 3e-3, 1e-4)
    assert gap(0, 0, 1.0, 1, 0.5, 1e-4) == 1
