"""Parity of the sm_103a library (through its C ABI) with the FP64 CPU oracle.

Bars (written out per test):
  * integer decisions (coordinate blocks, Floyd samples): bit-exact;
  * FP64 mode: relative Frobenius error of the iterate <= 1e-10 at every
    checked step;
  * FP32 storage with FP32 or 3xTF32 products: <= 1e-4 along the trajectory
    and |r_gpu - r_oracle| <= 0.1 tol on the final residual;
  * mixed (single-pass TF32 for the rank-q correction): residual agreement.
"""
import numpy as np
import pytest

import paper_1602_01768_gb300._binding as B
from oracle import oracle as orc
from paper_1602_01768_gb300 import workloads as wl

from gpu_util import empty_dev, export, from_dev, rel, stream_ptr, to_dev, torch_dtype

pytestmark = pytest.mark.gpu


def _handle(A, method, sketch, q, prec, seed=11, stream=0, core_fp64=0):
    n = A.shape[0]
    tdt = torch_dtype(prec)
    Ad = to_dev(A, tdt)
    opts = B.make_opts(method=method, sketch=sketch, q=q, prec=prec, seed=seed, stream_id=stream,
                       core_fp64=core_fp64)
    h = B.rbfgs_init(n, Ad.data_ptr(), n, prec == B.RB_FP64, opts, stream_ptr())
    return h


# --------------------------------------------------------------------------
# Sketch draws
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [B.RB_FP64, B.RB_FP32, B.RB_MIXED])
def test_gauss_sketch_bit_exact(prec):
    # the sketch is defined by binary32 operations in a fixed order, rounded to
    # TF32: the GPU draw equals the oracle's bit for bit in every precision
    for n, q, ks in ((1001, 24, (0, 1, 77, 2**31 + 5)), (4099, 128, (3,))):
        A = np.eye(n)
        h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=0xABCDEF12345, stream=3)
        try:
            for k in ks:
                out = empty_dev(n, q, torch_dtype(prec))
                B.rbfgs_draw_sketch(h, k, out.data_ptr(), n)
                S = from_dev(out)
                Sref = orc.gauss_sketch(0xABCDEF12345, 3, k, n, q)
                assert np.array_equal(S, Sref), (n, q, k, int(np.sum(S != Sref)))
        finally:
            B.rbfgs_destroy(h)


def test_coordinate_draws_bit_exact():
    n, q = 150, 16  # 10 blocks, the last one of size 6
    A, _, _ = wl.spd_spectrum(n, 1e3, 21)
    h = _handle(A, B.RB_METHOD_RBFGS, B.RB_SKETCH_COORD_TRACE, q, B.RB_FP64, seed=5, stream=1)
    try:
        for k in range(200):
            out = empty_dev(n, q, torch_dtype(B.RB_FP64))
            B.rbfgs_draw_sketch(h, k, out.data_ptr(), n)
            S = from_dev(out)
            b, first, size = orc.coord_trace_block(A, q, 5, 1, k)
            ref = np.zeros((n, q))
            ref[first + np.arange(size), np.arange(size)] = 1.0
            assert np.array_equal(S, ref), k
    finally:
        B.rbfgs_destroy(h)
    h = _handle(np.eye(97), B.RB_METHOD_ADARBFGS, B.RB_SKETCH_COORD_UNIFORM, 9, B.RB_FP64, seed=8, stream=2)
    try:
        for k in range(100):
            out = empty_dev(97, 9, torch_dtype(B.RB_FP64))
            B.rbfgs_draw_sketch(h, k, out.data_ptr(), 97)
            S = from_dev(out)
            idx = orc.floyd_sample(8, 2, k, orc.TAG_COORD, 97, 9)
            ref = np.zeros((97, 9))
            ref[idx, np.arange(9)] = 1.0
            assert np.array_equal(S, ref), k
    finally:
        B.rbfgs_destroy(h)


# --------------------------------------------------------------------------
# FP64 parity (<= 1e-10 relative Frobenius at every checked step)
# --------------------------------------------------------------------------
def test_rbfgs_fp64_c1_parity():
    w = wl.WORKLOADS["c1_rbfgs_fp64_n256"]
    A, _, _ = wl.c1_matrix()
    n, q = w["n"], w["q"]
    h = _handle(A, B.RB_METHOD_RBFGS, B.RB_SKETCH_GAUSS, q, B.RB_FP64, seed=w["seed"])
    X = np.eye(n)
    done = 0
    try:
        for chk in (1, 5, 50, 150, 300):
            B.rbfgs_step(h, chk - done)
            _, X = orc.rbfgs_run(A, X, q, orc.SKETCH_GAUSS, w["seed"], 0, done, chk - done)
            done = chk
            Xg = export(h, n, B.RB_FP64, B.RB_WHAT_X)
            assert rel(Xg, X) <= 1e-10, (chk, rel(Xg, X))
        r_gpu = B.rbfgs_residual(h, 0)
        r_orc = orc.residual(A, X)
        assert abs(r_gpu - r_orc) <= 1e-10 * max(r_orc, 1e-3)
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("n,q", [(203, 7), (64, 64), (1, 1)])
def test_rbfgs_fp64_ragged_parity(n, q):
    if n == 1:
        A = np.array([[2.5]])
    else:
        A, _, _ = wl.spd_spectrum(n, 50.0, 22)
    steps = 30 if n > 1 else 2
    h = _handle(A, B.RB_METHOD_RBFGS, B.RB_SKETCH_GAUSS, q, B.RB_FP64, seed=3)
    try:
        B.rbfgs_step(h, steps)
        _, X = orc.rbfgs_run(A, np.eye(n), q, orc.SKETCH_GAUSS, 3, 0, 0, steps)
        assert rel(export(h, n, B.RB_FP64, B.RB_WHAT_X), X) <= 1e-10
    finally:
        B.rbfgs_destroy(h)


def test_rbfgs_coordinate_fp64_parity():
    n, q = 150, 16
    A, _, _ = wl.spd_spectrum(n, 30.0, 23)
    h = _handle(A, B.RB_METHOD_RBFGS, B.RB_SKETCH_COORD_TRACE, q, B.RB_FP64, seed=6)
    try:
        B.rbfgs_step(h, 120)
        _, X = orc.rbfgs_run(A, np.eye(n), q, orc.SKETCH_COORD_TRACE, 6, 0, 0, 120)
        assert rel(export(h, n, B.RB_FP64, B.RB_WHAT_X), X) <= 1e-10
    finally:
        B.rbfgs_destroy(h)


# --------------------------------------------------------------------------
# Approximate inverse preconditioning, Eq. (BFGSas)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("sketch,kind,n,q", [(B.RB_SKETCH_GAUSS, orc.SKETCH_GAUSS, 256, 8),
                                             (B.RB_SKETCH_GAUSS, orc.SKETCH_GAUSS, 203, 7),
                                             (B.RB_SKETCH_COORD_TRACE, orc.SKETCH_COORD_TRACE, 150, 16)])
def test_aip_fp64_parity(sketch, kind, n, q):
    # relative Frobenius error of X against the FP64 oracle <= 1e-10 at every check
    A, _, _ = wl.spd_spectrum(n, 100.0, 41)
    h = _handle(A, B.RB_METHOD_AIP, sketch, q, B.RB_FP64, seed=9)
    X = np.eye(n)
    done = 0
    try:
        for chk in (1, 20, 150):
            B.aip_step(h, chk - done)
            _, X = orc.aip_run(A, X, q, kind, 9, 0, done, chk - done)
            done = chk
            assert rel(export(h, n, B.RB_FP64, B.RB_WHAT_X), X) <= 1e-10, chk
    finally:
        B.rbfgs_destroy(h)


def test_aip_fp32_parity_and_residual():
    # FP32 storage: <= 1e-4 relative along 60 steps (u = 6e-8 accumulated over the steps and
    # n-length dot products), and the library's exact residual matches the oracle's
    n, q = 512, 32
    A, _, _ = wl.spd_spectrum(n, 50.0, 42)
    h = _handle(A, B.RB_METHOD_AIP, B.RB_SKETCH_GAUSS, q, B.RB_FP32, seed=10)
    try:
        B.aip_step(h, 60)
        _, X = orc.aip_run(A, np.eye(n), q, orc.SKETCH_GAUSS, 10, 0, 0, 60)
        Xg = export(h, n, B.RB_FP32, B.RB_WHAT_X)
        assert rel(Xg, X) <= 1e-4
        r_gpu = B.rbfgs_residual(h, 0, 0)
        r_orc = orc.residual(A, X)
        assert abs(r_gpu - r_orc) <= 1e-3 * r_orc + 1e-6
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("sketch,kind", [(B.RB_SKETCH_GAUSS, orc.SKETCH_GAUSS),
                                         (B.RB_SKETCH_COORD_UNIFORM, orc.SKETCH_COORD_UNIFORM)])
def test_adarbfgs_fp64_parity(sketch, kind):
    n, q = 300, 12
    A, _, _ = wl.spd_spectrum(n, 100.0, 24)
    h = _handle(A, B.RB_METHOD_ADARBFGS, sketch, q, B.RB_FP64, seed=7)
    L = np.eye(n)
    done = 0
    try:
        for chk in (1, 10, 60):
            B.adarbfgs_step(h, chk - done)
            _, L = orc.adarbfgs_run(A, L, q, kind, 7, 0, done, chk - done)
            done = chk
            Lg = export(h, n, B.RB_FP64, B.RB_WHAT_L)
            assert rel(Lg, L) <= 1e-10, (chk, rel(Lg, L))
        Xg = export(h, n, B.RB_FP64, B.RB_WHAT_X)
        assert rel(Xg, L @ L.T) <= 1e-10
        assert abs(B.rbfgs_residual(h, 0) - orc.residual_factored(A, L)) <= 1e-10
        assert abs(B.rbfgs_residual(h, 40, 99) - orc.residual_sampled(A, 40, 99, L=L)) <= 1e-10
    finally:
        B.rbfgs_destroy(h)


# --------------------------------------------------------------------------
# FP32 storage: SIMT FP32 and tensor-core 3xTF32 products
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [B.RB_FP32, B.RB_TF32X3])
@pytest.mark.parametrize("n,q", [(1000, 64), (512, 32)])
def test_adarbfgs_fp32_parity(prec, n, q):
    # the oracle inverts the same FP32-rounded matrix the device holds
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    steps = 40
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=9)
    try:
        L = np.eye(n)
        done = 0
        for chk in (1, 10, steps):
            B.adarbfgs_step(h, chk - done)
            _, L = orc.adarbfgs_run(A, L, q, orc.SKETCH_GAUSS, 9, 0, done, chk - done)
            done = chk
            Lg = export(h, n, prec, B.RB_WHAT_L)
            assert rel(Lg, L) <= 1e-4, (chk, rel(Lg, L))
        r_orc = orc.residual_factored(A, L)
        r_gpu = B.rbfgs_residual(h, 0)
        assert abs(r_gpu - r_orc) <= 1e-3 * r_orc
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("n", [768, 2100])
def test_adarbfgs_tf32x3_one_step_from_general_L(n):
    # exercises the M-contiguous operand path (S = L S~ with L != I) and split-K; at n = 2100 the
    # products run stream-K (K >= 64 k-blocks) with ragged M and K, and W takes G's lo part from G's epilogue
    q = 64
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(4)
    L0 = np.eye(n) + 0.05 * rng.standard_normal((n, n))
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_TF32X3, seed=12)
    try:
        Ld = to_dev(L0, torch_dtype(B.RB_TF32X3))
        B.rbfgs_import(h, B.RB_WHAT_L, Ld.data_ptr(), n)
        B.rbfgs_set_step(h, 5)
        B.adarbfgs_step(h, 1)
        _, L1 = orc.adarbfgs_run(A, L0.astype(np.float32).astype(np.float64), q, orc.SKETCH_GAUSS, 12, 0, 5, 1)
        assert rel(export(h, n, B.RB_TF32X3, B.RB_WHAT_L), L1) <= 2e-5
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("n,q", [(1000, 64), (780, 32), (512, 128)])
def test_adarbfgs_mixed_one_step_from_general_L(n, q):
    # the single-pass TF32 persistent update kernel (ragged tiles when n % 128 != 0)
    n = n - (n % 4)  # TMA needs 16-byte rows
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(5)
    L0 = (np.eye(n) + 0.05 * rng.standard_normal((n, n))).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_MIXED, seed=14)
    try:
        Ld = to_dev(L0, torch_dtype(B.RB_MIXED))
        B.rbfgs_import(h, B.RB_WHAT_L, Ld.data_ptr(), n)
        B.rbfgs_set_step(h, 3)
        B.adarbfgs_step(h, 1)
        _, L1 = orc.adarbfgs_run(A, L0, q, orc.SKETCH_GAUSS, 14, 0, 3, 1)
        Lg = export(h, n, B.RB_MIXED, B.RB_WHAT_L)
        # single-pass TF32 on the correction S^ V only: error ~ 2^-11 |S^ V|,
        # so relative to L the bound scales with |L1 - L0| / |L1|
        corr = rel(Lg - L0, L1 - L0)
        assert corr <= 2e-3
        assert rel(Lg, L1) <= 2e-3 * np.linalg.norm(L1 - L0) / np.linalg.norm(L1) + 1e-5
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("n,q", [(2100, 64), (2052, 128)])
def test_adarbfgs_mixed_two_steps_streamk_ragged(n, q):
    # sizes where the GEMMs run stream-K (pieces of a tile added by the CTA that finishes it) and
    # several CTAs share each row block of the fused update (their S_next pieces added likewise),
    # with ragged M and K; the second step takes S and S's lo part from the first step's fused kernel
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(6)
    L0 = (np.eye(n) + 0.05 * rng.standard_normal((n, n))).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_MIXED, seed=15)
    try:
        Ld = to_dev(L0, torch_dtype(B.RB_MIXED))
        B.rbfgs_import(h, B.RB_WHAT_L, Ld.data_ptr(), n)
        B.rbfgs_set_step(h, 7)
        B.adarbfgs_step(h, 2)
        _, L2 = orc.adarbfgs_run(A, L0, q, orc.SKETCH_GAUSS, 15, 0, 7, 2)
        Lg = export(h, n, B.RB_MIXED, B.RB_WHAT_L)
        # single-pass TF32 corrections: error ~ 2^-11 of each step's correction
        assert rel(Lg - L0, L2 - L0) <= 3e-3
        assert rel(Lg, L2) <= 3e-3 * np.linalg.norm(L2 - L0) / np.linalg.norm(L2) + 1e-5
    finally:
        B.rbfgs_destroy(h)


def test_adarbfgs_mixed_reaches_tolerance_like_oracle():
    n, q, tol = 512, 32, 1e-4
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_MIXED, seed=13)
    try:
        st, iters, r = B.rbfgs_solve(h, tol, 3000, 16, 128, 0)
        assert st == B.RB_OK and r <= tol
        _, L = orc.adarbfgs_run(A, np.eye(n), q, orc.SKETCH_GAUSS, 13, 0, 0, iters)
        r_orc = orc.residual_factored(A, L)
        Lg = export(h, n, B.RB_MIXED, B.RB_WHAT_L)
        r_gpu_in_fp64 = orc.residual_factored(A, Lg)
        # final-residual agreement after the same number of steps: |r_gpu - r_oracle| <= 0.1 tol,
        # both evaluated exactly in FP64 by the oracle
        assert abs(r_gpu_in_fp64 - r_orc) <= 0.1 * tol, (r_gpu_in_fp64, r_orc, iters)
        assert r_gpu_in_fp64 <= 1.1 * tol
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("prec", [B.RB_TF32X3, B.RB_MIXED])
def test_adarbfgs_fp64_core_with_fp32_storage(prec):
    # opts.core_fp64 = 1: the q x q Cholesky factors and their inverses in FP64 on the side stream.
    # Same bars as the FP32-core forms: 3xTF32 <= 1e-4 along the trajectory; mixed within the
    # single-pass correction's error.  The FP64 and FP32 cores differ only by the FP32 rounding of
    # a well-conditioned q x q factorisation.
    n, q = 512, 32
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    h64 = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=17, core_fp64=1)
    h32 = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=17, core_fp64=-1)
    try:
        L = np.eye(n)
        done = 0
        for chk in (1, 10, 40):
            B.adarbfgs_step(h64, chk - done)
            B.adarbfgs_step(h32, chk - done)
            _, Ln = orc.adarbfgs_run(A, L, q, orc.SKETCH_GAUSS, 17, 0, done, chk - done)
            L64 = export(h64, n, prec, B.RB_WHAT_L)
            L32 = export(h32, n, prec, B.RB_WHAT_L)
            # mixed: the single-pass correction leaves ~2^-11 of each step's change (2.3e-3 of L
            # after 10 steps at this size), hence 1.5e-2 over 40 steps
            bar = 1e-4 if prec == B.RB_TF32X3 else 1.5e-2
            assert rel(L64, Ln) <= bar, (chk, rel(L64, Ln))
            # mixed: the two runs drift apart like two mixed runs of the oracle would, by the
            # single-pass correction's rounding (1.7e-3 after 40 steps measured)
            assert rel(L64, L32) <= (1e-4 if prec == B.RB_TF32X3 else 1e-2), (chk, rel(L64, L32))
            L, done = Ln, chk
        r_orc = orc.residual_factored(A, L)
        r64 = orc.residual_factored(A, export(h64, n, prec, B.RB_WHAT_L))
        assert abs(r64 - r_orc) <= (1e-3 if prec == B.RB_TF32X3 else 5e-2) * r_orc
    finally:
        B.rbfgs_destroy(h64)
        B.rbfgs_destroy(h32)


def test_adarbfgs_tf32_single_pass_parity():
    # RB_TF32: every tensor-core product in one TF32 pass (unit roundoff 2^-11 ~ 4.9e-4 per
    # product).  Bar: relative Frobenius error of L <= 2e-2 after 10 and 30 steps, and the exact
    # residual of the device factor within 5e-2 relative of the oracle's.
    n, q = 512, 32
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_TF32, seed=18)
    try:
        L = np.eye(n)
        done = 0
        for chk in (10, 30):
            B.adarbfgs_step(h, chk - done)
            _, L = orc.adarbfgs_run(A, L, q, orc.SKETCH_GAUSS, 18, 0, done, chk - done)
            done = chk
            Lg = export(h, n, B.RB_TF32, B.RB_WHAT_L)
            assert rel(Lg, L) <= 2e-2, (chk, rel(Lg, L))
        r_orc = orc.residual_factored(A, L)
        assert abs(orc.residual_factored(A, Lg) - r_orc) <= 5e-2 * r_orc
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("prec", [B.RB_MIXED, B.RB_TF32X3, B.RB_BF16X3])
def test_adarbfgs_cols_tensor_core_parity(prec):
    # AdaRBFGS_cols (q uniform distinct coordinates, Sec. 10) through the tensor-core step: S = L[:, C]
    # is a gather (exact) and S~^T S~ = I, so D = I.  Two steps from a general L: 3xTF32 <= 2e-5;
    # mixed and BF16x3 within 3e-3 of the change (single-pass correction).
    n, q = 1024, 32
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(8)
    L0 = (np.eye(n) + 0.05 * rng.standard_normal((n, n))).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_COORD_UNIFORM, q, prec, seed=19)
    try:
        Ld = to_dev(L0, torch_dtype(prec))
        B.rbfgs_import(h, B.RB_WHAT_L, Ld.data_ptr(), n)
        B.rbfgs_set_step(h, 4)
        B.adarbfgs_step(h, 2)
        _, L2 = orc.adarbfgs_run(A, L0, q, orc.SKETCH_COORD_UNIFORM, 19, 0, 4, 2)
        Lg = export(h, n, prec, B.RB_WHAT_L)
        if prec == B.RB_TF32X3:
            assert rel(Lg, L2) <= 2e-5, rel(Lg, L2)
        else:
            assert rel(Lg - L0, L2 - L0) <= 3e-3, rel(Lg - L0, L2 - L0)
        # and a run from L0 = I converges like the oracle's
        B.rbfgs_reset(h, 19, 0)
        B.adarbfgs_step(h, 60)
        _, L60 = orc.adarbfgs_run(A, np.eye(n), q, orc.SKETCH_COORD_UNIFORM, 19, 0, 0, 60)
        r_orc = orc.residual_factored(A, L60)
        r_gpu = orc.residual_factored(A, export(h, n, prec, B.RB_WHAT_L))
        assert abs(r_gpu - r_orc) <= 1e-2 * r_orc, (r_gpu, r_orc)
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("sketch,kind,q", [(B.RB_SKETCH_GAUSS, orc.SKETCH_GAUSS, 32),
                                           (B.RB_SKETCH_COORD_TRACE, orc.SKETCH_COORD_TRACE, 16)])
def test_rbfgs_fp32_parity(sketch, kind, q):
    # RBFGS with FP32 storage and products: <= 1e-4 relative along 40 steps (u = 6e-8 accumulated
    # over the steps and n-length dot products), residual within 1e-3 relative
    n = 512
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_RBFGS, sketch, q, B.RB_FP32, seed=20)
    try:
        X = np.eye(n)
        done = 0
        for chk in (1, 10, 40):
            B.rbfgs_step(h, chk - done)
            _, X = orc.rbfgs_run(A, X, q, kind, 20, 0, done, chk - done)
            done = chk
            Xg = export(h, n, B.RB_FP32, B.RB_WHAT_X)
            assert rel(Xg, X) <= 1e-4, (chk, rel(Xg, X))
        r_orc = orc.residual(A, X)
        assert abs(B.rbfgs_residual(h, 0) - r_orc) <= 1e-3 * r_orc
    finally:
        B.rbfgs_destroy(h)


# --------------------------------------------------------------------------
# Tensor-core RBFGS (Eq. (qunac)) and AIP (Eq. (BFGSas)) steps
# --------------------------------------------------------------------------
# Bars: 3xTF32 products <= 1e-4 relative along 40 steps (~FP32 accuracy); mixed (the rank-2q or
# rank-q update in one TF32 pass: it vanishes at the fixed point, so its 2^-11 rounding scales
# with the step's change) <= 1.5e-2; single-pass TF32 <= 2e-2.
_X_BARS = {B.RB_TF32X3: 1e-4, B.RB_MIXED: 1.5e-2, B.RB_TF32: 2e-2}


@pytest.mark.parametrize("prec", [B.RB_TF32X3, B.RB_MIXED, B.RB_TF32])
@pytest.mark.parametrize("n,q", [(512, 32), (1028, 64)])
def test_rbfgs_tensor_core_parity(prec, n, q):
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_RBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=24)
    try:
        X = np.eye(n)
        done = 0
        for chk in (1, 10, 40):
            B.rbfgs_step(h, chk - done)
            _, X = orc.rbfgs_run(A, X, q, orc.SKETCH_GAUSS, 24, 0, done, chk - done)
            done = chk
            Xg = export(h, n, prec, B.RB_WHAT_X)
            assert rel(Xg, X) <= _X_BARS[prec], (chk, rel(Xg, X))
            assert rel(Xg, Xg.T) <= 1e-5  # the rank-2q update keeps X symmetric up to rounding
        r_orc = orc.residual(A, X)
        assert abs(orc.residual(A, Xg) - r_orc) <= (1e-3 if prec == B.RB_TF32X3 else 5e-2) * r_orc
    finally:
        B.rbfgs_destroy(h)


def test_rbfgs_mixed_reaches_tolerance_like_oracle():
    # a well-conditioned matrix (kappa = 10), n = 256, q = 32: the mixed tensor-core RBFGS reaches
    # 1e-4 and its iterate, evaluated exactly in FP64, is within 0.1 tol of the oracle's
    n, q, tol = 256, 32, 1e-4
    A, _, _ = wl.spd_spectrum(n, 10.0, 43)
    A = A.astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_RBFGS, B.RB_SKETCH_GAUSS, q, B.RB_MIXED, seed=25)
    try:
        st, iters, r = B.rbfgs_solve(h, tol, 5000, 16, 0, 0)
        assert st == B.RB_OK and r <= tol
        _, X = orc.rbfgs_run(A, np.eye(n), q, orc.SKETCH_GAUSS, 25, 0, 0, iters)
        r_orc = orc.residual(A, X)
        r_gpu = orc.residual(A, export(h, n, B.RB_MIXED, B.RB_WHAT_X))
        assert abs(r_gpu - r_orc) <= 0.1 * tol, (r_gpu, r_orc, iters)
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("prec", [B.RB_TF32X3, B.RB_MIXED])
def test_aip_tensor_core_parity(prec):
    n, q = 512, 32
    A, _, _ = wl.spd_spectrum(n, 50.0, 44)
    A = A.astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_AIP, B.RB_SKETCH_GAUSS, q, prec, seed=26)
    try:
        X = np.eye(n)
        done = 0
        for chk in (1, 10, 40):
            B.aip_step(h, chk - done)
            _, X = orc.aip_run(A, X, q, orc.SKETCH_GAUSS, 26, 0, done, chk - done)
            done = chk
            assert rel(export(h, n, prec, B.RB_WHAT_X), X) <= _X_BARS[prec], chk
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("method,kind,step", [(B.RB_METHOD_RBFGS, "rbfgs", B.rbfgs_step),
                                              (B.RB_METHOD_AIP, "aip", B.aip_step)])
def test_coordinate_tensor_core_parity(method, kind, step):
    # trace-weighted coordinate blocks (bit-exact draws); the one pass over X (Y = X A[:, C], or
    # W^T = X^T A[:, C]) on the tensor cores in 3 terms: <= 1e-4 along 100 steps
    n, q = 512, 16
    A, _, _ = wl.spd_spectrum(n, 30.0, 45)
    A = A.astype(np.float32).astype(np.float64)
    h = _handle(A, method, B.RB_SKETCH_COORD_TRACE, q, B.RB_TF32X3, seed=27)
    run = orc.rbfgs_run if kind == "rbfgs" else orc.aip_run
    try:
        step(h, 100)
        _, X = run(A, np.eye(n), q, orc.SKETCH_COORD_TRACE, 27, 0, 0, 100)
        assert rel(export(h, n, B.RB_TF32X3, B.RB_WHAT_X), X) <= 1e-4
    finally:
        B.rbfgs_destroy(h)


# --------------------------------------------------------------------------
# BF16-split forms: G = A S and W^T = L^T G as kind::f16 products
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,q", [(768, 64), (4100, 128)])
def test_adarbfgs_bf16x3_one_step_from_general_L(n, q):
    # 3-term BF16 splits carry ~2^-16 relative error per product (x = hi + lo to 2^-17, the
    # dropped lo lo term 2^-16); the rank-q correction is single-pass TF32 as in the mixed form,
    # so the step's change is within 3e-3 of the oracle's.  At n = 4100 the BF16 GEMMs run
    # stream-K (65 k-blocks of 64 per tile) with ragged M and K.
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(9)
    L0 = (np.eye(n) + 0.05 * rng.standard_normal((n, n))).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_BF16X3, seed=21)
    try:
        Ld = to_dev(L0, torch_dtype(B.RB_BF16X3))
        B.rbfgs_import(h, B.RB_WHAT_L, Ld.data_ptr(), n)
        B.rbfgs_set_step(h, 2)
        B.adarbfgs_step(h, 2)
        _, L2 = orc.adarbfgs_run(A, L0, q, orc.SKETCH_GAUSS, 21, 0, 2, 2)
        Lg = export(h, n, B.RB_BF16X3, B.RB_WHAT_L)
        corr = rel(Lg - L0, L2 - L0)
        assert corr <= 3e-3, corr
    finally:
        B.rbfgs_destroy(h)


def test_adarbfgs_bf16x3_reaches_tolerance_like_oracle():
    # the n x n sparse ridge-Hessian recipe of the n = 16384 workload at n = 1024 (kappa ~ 10):
    # the BF16x3 form reaches tol 1e-4 and its factor, evaluated exactly in FP64, is within
    # 0.1 tol of the oracle's after the same number of steps
    n, q, tol = 1024, 32, 1e-4
    A = wl.c3_matrix(n=n).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_BF16X3, seed=22)
    try:
        st, iters, r = B.rbfgs_solve(h, tol, 5000, 16, 256, 0)
        assert st == B.RB_OK and r <= tol
        _, L = orc.adarbfgs_run(A, np.eye(n), q, orc.SKETCH_GAUSS, 22, 0, 0, iters)
        r_orc = orc.residual_factored(A, L)
        r_gpu = orc.residual_factored(A, export(h, n, B.RB_BF16X3, B.RB_WHAT_L))
        assert abs(r_gpu - r_orc) <= 0.1 * tol, (r_gpu, r_orc, iters)
        assert r_gpu <= 1.1 * tol
    finally:
        B.rbfgs_destroy(h)


def test_adarbfgs_bf16_single_pass_parity():
    # RB_BF16: G and W^T in one BF16 pass (unit roundoff 2^-8 per operand), the rest single-pass
    # TF32.  Bar: relative Frobenius error of L <= 1e-1 after 10 and 30 steps, the exact residual
    # within 2e-1 relative of the oracle's.
    n, q = 512, 32
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_BF16, seed=23)
    try:
        L = np.eye(n)
        done = 0
        for chk in (10, 30):
            B.adarbfgs_step(h, chk - done)
            _, L = orc.adarbfgs_run(A, L, q, orc.SKETCH_GAUSS, 23, 0, done, chk - done)
            done = chk
            Lg = export(h, n, B.RB_BF16, B.RB_WHAT_L)
            assert rel(Lg, L) <= 1e-1, (chk, rel(Lg, L))
        r_orc = orc.residual_factored(A, L)
        assert abs(orc.residual_factored(A, Lg) - r_orc) <= 2e-1 * r_orc
    finally:
        B.rbfgs_destroy(h)


def test_bf16_forms_rejected_where_not_built():
    A = to_dev(np.eye(64), torch_dtype(B.RB_BF16X3))
    for method in (B.RB_METHOD_RBFGS, B.RB_METHOD_AIP):
        with pytest.raises(B.RbfgsError) as e:
            B.rbfgs_init(64, A.data_ptr(), 64, False, B.make_opts(method=method, q=8, prec=B.RB_BF16X3), 0)
        assert e.value.status == B.RB_EUNSUPPORTED
    with pytest.raises(B.RbfgsError) as e:
        B.newton_schulz_init(64, A.data_ptr(), 64, False, B.RB_BF16X3, 0, 1.0, 0)
    assert e.value.status == B.RB_EUNSUPPORTED


# --------------------------------------------------------------------------
# Comparison methods
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec,tol", [(B.RB_FP64, 1e-10), (B.RB_FP32, 1e-4), (B.RB_TF32X3, 1e-4)])
def test_newton_schulz_parity(prec, tol):
    n = 384
    A, _, lam = wl.spd_spectrum(n, 30.0, 25)
    Ad = to_dev(A, torch_dtype(prec))
    h = B.newton_schulz_init(n, Ad.data_ptr(), n, prec == B.RB_FP64, prec, 0, float(lam.max()), stream_ptr())
    try:
        X = orc.ns_init(A, float(lam.max()))
        for _ in range(3):
            B.newton_schulz_step(h, 4)
            for _ in range(4):
                X = orc.ns_step(A, X)
            assert rel(export(h, n, prec, B.RB_WHAT_X), X) <= tol
    finally:
        B.rbfgs_destroy(h)


def test_newton_schulz_power_iteration_sigma():
    n = 200
    A, _, lam = wl.spd_spectrum(n, 10.0, 26)
    Ad = to_dev(A, torch_dtype(B.RB_FP64))
    h = B.newton_schulz_init(n, Ad.data_ptr(), n, True, B.RB_FP64, 60, 0.0, stream_ptr())
    try:
        assert abs(B.rbfgs_sigma(h) - orc.power_norm(A, 60)) <= 1e-12 * lam.max()
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("prec,tol", [(B.RB_FP64, 1e-10), (B.RB_FP32, 1e-4)])
def test_mr_parity(prec, tol):
    n = 256
    A, _, _ = wl.spd_spectrum(n, 20.0, 27)
    Ad = to_dev(A, torch_dtype(prec))
    h = B.mr_init(n, Ad.data_ptr(), n, prec == B.RB_FP64, prec, stream_ptr())
    try:
        X = orc.mr_init(A)
        assert rel(export(h, n, prec, B.RB_WHAT_X), X) <= tol
        B.mr_step(h, 5)
        for _ in range(5):
            _, X = orc.mr_step(A, X)
        assert rel(export(h, n, prec, B.RB_WHAT_X), X) <= tol
    finally:
        B.rbfgs_destroy(h)


# --------------------------------------------------------------------------
# Failure paths, checkpoint / resume
# --------------------------------------------------------------------------
def test_indefinite_matrix_reports_notspd_and_keeps_iterate():
    n, q = 40, 4
    A = -np.eye(n)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_FP64)
    try:
        B.adarbfgs_step(h, 3)
        with pytest.raises(B.RbfgsError) as e:
            B.rbfgs_sync(h)
        assert e.value.status == B.RB_ENOTSPD
        assert np.array_equal(export(h, n, B.RB_FP64, B.RB_WHAT_L), np.eye(n))
    finally:
        B.rbfgs_destroy(h)


def test_bounded_wait_runs_out_and_leaves_the_iterate():
    # a kernel waits on an mbarrier that nothing completes (no copy or MMA in flight) with a limit
    # of 2e6 SM cycles (about a millisecond): the wait gives up, the handle's status word records the
    # timeout, later steps leave L untouched, the next synchronising call reports RB_ETIMEOUT, and a
    # fresh handle on the same device then steps normally
    n, q = 256, 32
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_MIXED, seed=28)
    try:
        B.adarbfgs_step(h, 3)
        B.rbfgs_sync(h)
        L0 = export(h, n, B.RB_MIXED, B.RB_WHAT_L)
        B.rbfgs_wait_selftest(h, 2_000_000)
        B.adarbfgs_step(h, 2)
        with pytest.raises(B.RbfgsError) as e:
            B.rbfgs_sync(h)
        assert e.value.status == B.RB_ETIMEOUT
        assert np.array_equal(export(h, n, B.RB_MIXED, B.RB_WHAT_L), L0)
    finally:
        B.rbfgs_destroy(h)
    h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, B.RB_MIXED, seed=28)
    try:
        B.adarbfgs_step(h, 3)
        B.rbfgs_sync(h)
        assert np.array_equal(export(h, n, B.RB_MIXED, B.RB_WHAT_L), L0)  # the same three steps
    finally:
        B.rbfgs_destroy(h)
    with pytest.raises(B.RbfgsError) as e:
        B.rbfgs_wait_selftest(None, 10)
    assert e.value.status == B.RB_EINVAL


def test_invalid_arguments_are_rejected():
    with pytest.raises(B.RbfgsError) as e:
        B.rbfgs_init(0, 1, 1, 0, B.make_opts(), 0)
    assert e.value.status == B.RB_EINVAL
    A = to_dev(np.eye(8), torch_dtype(B.RB_FP64))
    with pytest.raises(B.RbfgsError):
        B.rbfgs_init(8, A.data_ptr(), 8, 1, B.make_opts(q=9), 0)


@pytest.mark.parametrize("prec", [B.RB_BF16X3, B.RB_BF16, B.RB_MIXED, B.RB_TF32X3])
def test_repeated_runs_are_bit_identical(prec):
    # Two handles with the same seed run the same steps: every kernel sums in a fixed order, so the
    # factors agree bit for bit.  At n = 3000 A and L stay in L2, the GEMM rings wrap several times per
    # CTA and refills land fast: a slot released before its reader is done shows up here as a
    # difference (an early A-slot release in the BF16 GEMM did, at n = 6544, as a stalled solve).
    n, q, K = 3000, 64, 24
    A = wl.c2_matrix(n=n).astype(np.float32).astype(np.float64)
    out = []
    for _ in range(2):
        h = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=41)
        try:
            B.adarbfgs_step(h, K)
            out.append(export(h, n, prec, B.RB_WHAT_L))
        finally:
            B.rbfgs_destroy(h)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", [B.RB_FP64, B.RB_TF32X3, B.RB_MIXED, B.RB_BF16X3])
def test_checkpoint_resume_is_bit_exact(prec):
    # (mixed: the resumed handle forms S with the fused kernel's update-free pass, the uninterrupted
    # one takes S from the previous fused update -- the same arithmetic path, so the same bits)
    n, q, K = 256, 16, 12
    A = wl.c2_matrix(n=n)
    tdt = torch_dtype(prec)
    h1 = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=31)
    h2 = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=31)
    try:
        B.adarbfgs_step(h1, 2 * K)
        B.adarbfgs_step(h2, K)
        ck = empty_dev(n, n, tdt)
        B.rbfgs_export(h2, B.RB_WHAT_L, ck.data_ptr(), n)
        k = B.rbfgs_get_step(h2)
        B.rbfgs_destroy(h2)
        h2 = _handle(A, B.RB_METHOD_ADARBFGS, B.RB_SKETCH_GAUSS, q, prec, seed=31)
        B.rbfgs_import(h2, B.RB_WHAT_L, ck.data_ptr(), n)
        B.rbfgs_set_step(h2, k)
        B.adarbfgs_step(h2, K)
        assert np.array_equal(export(h1, n, prec, B.RB_WHAT_L), export(h2, n, prec, B.RB_WHAT_L))
    finally:
        B.rbfgs_destroy(h1)
        B.rbfgs_destroy(h2)


def test_fp64_core_on_a_cluster_matches_one_cta_and_the_oracle():
    # The q x q core of Algorithm 4 in FP64 (C C^T = sym(M), written as C^-T): spread over a cluster
    # of 8 CTAs it gives the same bits as on one CTA (each element is computed by one thread in the
    # same order), and C^-T agrees with the oracle's FP64 Cholesky factor inverted by Gauss-Jordan
    # to FP32 rounding.  An indefinite M returns RB_ENOTSPD and leaves the output untouched.
    import torch

    rng = np.random.default_rng(5)
    for q in (128, 100, 64, 33, 7):
        Z = rng.standard_normal((4 * q, q))
        M = (Z.T @ Z / (4 * q) + 1e-3 * np.eye(q)).astype(np.float32)
        Md = to_dev(M, torch.float32)
        outs = {}
        for cl in (1, 8):
            out = empty_dev(q, q, torch.float32)
            used = B.rbfgs_core64(q, Md.data_ptr(), -1.0, out.data_ptr(), q, cl, stream_ptr())
            outs[cl] = (used, from_dev(out))
        assert outs[1][0] == 1 and outs[8][0] == 8, (outs[1][0], outs[8][0])
        assert np.array_equal(outs[1][1], outs[8][1]), q
        rc, Cf = orc.cholesky(M.astype(np.float64))
        assert rc == 0
        ref = -orc.gauss_jordan(Cf).T
        assert rel(outs[8][1], ref) <= 1e-6, (q, rel(outs[8][1], ref))
    q = 48
    M = np.eye(q, dtype=np.float32)
    M[3, 5] = M[5, 3] = 2.0  # the 2 x 2 block [[1, 2], [2, 1]] is indefinite
    Md = to_dev(M, torch.float32)
    out = empty_dev(q, q, torch.float32)
    out.fill_(7.0)
    with pytest.raises(B.RbfgsError):
        B.rbfgs_core64(q, Md.data_ptr(), 1.0, out.data_ptr(), q, 8, stream_ptr())
    assert np.all(from_dev(out) == 7.0)
