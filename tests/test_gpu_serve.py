"""Serving loop with continuous batching: each request's result is the same
alone and in a mix of concurrent requests, admission respects the HBM budget,
and the returned factor meets the tolerance when checked in FP64 by the oracle."""
import numpy as np
import pytest

import paper_1602_01768_gb300._binding as B
from oracle import oracle as orc
from paper_1602_01768_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _req(n, seed):
    import torch

    A = wl.c5_matrix(n, seed).astype(np.float32)
    A_host = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()  # column-major, symmetric anyway
    out = torch.zeros(n, n, dtype=torch.float32).pin_memory()
    return A, A_host, out


def _submit(s, A_host, out, n, tol, seed):
    return B.rb_srv_submit(s, n, A_host.data_ptr(), False, n, False, tol, seed, 0, out.data_ptr(), False, n)


def test_result_same_alone_and_in_the_mix():
    tol = 1e-4
    sizes = [(384, 51), (256, 52), (512, 53), (320, 54), (448, 55), (288, 56)]
    reqs = [_req(n, sd) for n, sd in sizes]
    s = B.rb_srv_create(8 << 30, 8, B.RB_MIXED, 16, 128, 20000)
    try:
        # alone
        A0, A0h, out_alone = reqs[0]
        t = _submit(s, A0h, out_alone, sizes[0][0], tol, 1000)
        r_alone = B.rb_srv_wait(s, t)
        assert r_alone.status == B.RB_OK and r_alone.resid <= tol
        L_alone = out_alone.numpy().T.copy()
        # the same request in a mix of six submitted back to back
        outs = [np.zeros(0)] * len(reqs)
        tickets = []
        import torch

        mix_out0 = torch.zeros_like(out_alone).pin_memory()
        for i, ((n, sd), (A, Ah, out)) in enumerate(zip(sizes, reqs)):
            o = mix_out0 if i == 0 else out
            tickets.append(_submit(s, Ah, o, n, tol, 1000 if i == 0 else 2000 + i))
        res = [B.rb_srv_wait(s, t) for t in tickets]
        assert all(r.status == B.RB_OK for r in res)
        L_mix = mix_out0.numpy().T.copy()
        assert res[0].iters == r_alone.iters
        assert np.array_equal(L_mix, L_alone)
        st = B.rb_srv_stats(s)
        assert st.completed == 7 and st.failed == 0 and st.p99_s >= st.p50_s > 0
        # FP64 check of a returned factor against the oracle's residual definition
        L = L_alone.astype(np.float64)
        assert orc.residual_factored(A0.astype(np.float64), L) <= 1.2 * tol
    finally:
        B.rb_srv_destroy(s)


def test_admission_respects_budget_and_every_request_finishes():
    tol = 1e-3
    n = 256
    opts = B.make_opts(method=B.RB_METHOD_ADARBFGS, q=32, prec=B.RB_MIXED)
    one = B.rbfgs_footprint(n, opts) + 4 * n * n  # plus the host staging copy
    s = B.rb_srv_create(int(1.5 * one), 8, B.RB_MIXED, 16, 64, 20000)  # room for one request at a time
    try:
        reqs = [_req(n, 60 + i) for i in range(4)]
        tickets = [_submit(s, Ah, out, n, tol, 70 + i) for i, (A, Ah, out) in enumerate(reqs)]
        res = [B.rb_srv_wait(s, t) for t in tickets]
        assert all(r.status == B.RB_OK and r.resid <= tol for r in res)
        # one at a time: each later request waited for the previous one
        assert res[3].queue_s >= res[0].latency_s * 0.5
    finally:
        B.rb_srv_destroy(s)


def test_oversize_request_is_rejected():
    s = B.rb_srv_create(1 << 20, 4)
    try:
        with pytest.raises(B.RbfgsError) as e:
            B.rb_srv_submit(s, 4096, 1, True, 4096, False, 1e-4, 0)
        assert e.value.status == B.RB_ENOMEM
    finally:
        B.rb_srv_destroy(s)


def test_form_per_tolerance_and_floor_limited_requests():
    # a BF16x3 server runs tol >= 1e-4 in BF16x3 and smaller tolerances in the 3xTF32 mixed form; a
    # tolerance below what FP32 storage reaches (1e-9) finishes as floor-limited (RB_NOTCONV) well
    # before max_iter, with the floor it reached, which the oracle confirms in FP64
    n = 384
    s = B.rb_srv_create(8 << 30, 8, B.RB_BF16X3, 16, 128, 20000)
    try:
        A, Ah, out = _req(n, 81)
        _, Ah2, out2 = _req(n, 81)
        t1 = _submit(s, Ah, out, n, 1e-4, 90)
        t2 = _submit(s, Ah2, out2, n, 1e-9, 91)
        r1, r2 = B.rb_srv_wait(s, t1), B.rb_srv_wait(s, t2)
        assert r1.status == B.RB_OK and r1.prec == B.RB_BF16X3 and not r1.floor_limited
        assert r2.status == B.RB_NOTCONV and r2.prec == B.RB_MIXED and r2.floor_limited
        assert r2.iters < 20000 and r2.resid < 1e-4
        r64 = orc.residual_factored(A.astype(np.float64), out2.numpy().T.astype(np.float64))
        assert r64 <= 3 * r2.resid, (r64, r2.resid)
    finally:
        B.rb_srv_destroy(s)
