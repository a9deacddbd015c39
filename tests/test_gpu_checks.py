"""Residual-check scheduling: the predicted spacing (check_every < 0) stops a
solve within a check spacing of where checks every e steps stop it, with a
factor that meets the tolerance in FP64."""
import numpy as np
import pytest

import paper_1602_01768_gb300._binding as B
from oracle import oracle as orc
from paper_1602_01768_gb300 import workloads as wl

from gpu_util import export, stream_ptr, to_dev, torch_dtype

pytestmark = pytest.mark.gpu


def _handle(A, q, prec, seed):
    n = A.shape[0]
    Ad = to_dev(A, torch_dtype(prec))
    o = B.make_opts(method=B.RB_METHOD_ADARBFGS, sketch=B.RB_SKETCH_GAUSS, q=q, prec=prec, seed=seed)
    return B.rbfgs_init(n, Ad.data_ptr(), n, False, o, stream_ptr()), Ad


@pytest.mark.parametrize("prec", [B.RB_MIXED, B.RB_BF16X3])
def test_predicted_spacing_stops_near_the_fixed_schedule(prec):
    n, q, tol, e = 1024, 32, 1e-4, 16
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    out = {}
    for mode in (e, -e):
        h, _Ad = _handle(A, q, prec, 21)
        try:
            st, iters, r = B.rbfgs_solve(h, tol, 20000, mode, 256, 0)  # exact confirmation
            L = export(h, n, prec, B.RB_WHAT_L)
        finally:
            B.rbfgs_destroy(h)
        assert st == B.RB_OK and r <= tol, (mode, st, r)
        out[mode] = (iters, r, L)
    it_f, it_p = out[e][0], out[-e][0]
    # both schedules see the same iterates; each stops at its first check below tol (a fresh column
    # sample per check, an exact confirmation), so they stop within two spacings of each other
    assert abs(it_p - it_f) <= 2 * e, (it_f, it_p)
    assert orc.residual_factored(A, out[-e][2]) <= tol
