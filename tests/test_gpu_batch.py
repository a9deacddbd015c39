"""Batched coordinate RBFGS (one persistent launch for many uneven problems):
parity with the FP64 oracle per problem, independence from the batch's
composition, and the solve loop."""
import numpy as np
import pytest

import paper_1602_01768_gb300._binding as B
from oracle import oracle as orc
from paper_1602_01768_gb300 import workloads as wl

from gpu_util import empty_dev, from_dev, rel, stream_ptr, to_dev

pytestmark = pytest.mark.gpu


def _problems(count, seed, nmax=220):
    out = []
    for A, q, kappa in wl.c4_problems(count=count * 4, seed=seed):
        if A.shape[0] <= nmax:
            out.append((A.astype(np.float32).astype(np.float64), q, kappa))
        if len(out) == count:
            break
    return out


def _create(probs, seed, stream_ids=None):
    import torch

    devs = [to_dev(A, torch.float32) for A, _, _ in probs]
    n = [A.shape[0] for A, _, _ in probs]
    b = B.rb_batch_create(n, [d.data_ptr() for d in devs], n, False, [q for _, q, _ in probs], seed,
                          stream_ids=stream_ids, stream=stream_ptr())
    return b, n


def _export(b, i, n):
    import torch

    out = empty_dev(n, n, torch.float32)
    B.rb_batch_export(b, i, out.data_ptr(), n)
    return from_dev(out)


def test_batch_matches_oracle_per_problem():
    probs = _problems(8, 4)
    seed, steps = 77, 60
    b, n = _create(probs, seed)
    try:
        B.rb_batch_step(b, steps)
        for i, (A, q, _) in enumerate(probs):
            _, X = orc.rbfgs_run(A, np.eye(n[i]), q, orc.SKETCH_COORD_TRACE, seed, i, 0, steps)
            assert rel(_export(b, i, n[i]), X) <= 1e-4, (i, n[i], q)
    finally:
        B.rb_batch_destroy(b)


def test_batch_result_is_independent_of_the_mix():
    probs = _problems(10, 5)
    b, n = _create(probs, 9)
    b1, n1 = _create([probs[3]], 9, stream_ids=[3])
    try:
        B.rb_batch_step(b, 25)
        B.rb_batch_step(b1, 25)
        assert np.array_equal(_export(b, 3, n[3]), _export(b1, 0, n1[0]))
    finally:
        B.rb_batch_destroy(b)
        B.rb_batch_destroy(b1)


def test_batch_solve_converges_and_residual_is_honest():
    # well-conditioned problems so that coordinate RBFGS reaches the tolerance quickly
    probs = []
    for i, n in enumerate((40, 72, 128, 36, 100)):
        A, _, _ = wl.spd_spectrum(n, 3.0, 300 + i)
        probs.append((A.astype(np.float32).astype(np.float64), (4, 8, 16, 32, 8)[i], 3.0))
    b, n = _create(probs, 21)
    try:
        rc, iters, resid, status, nconv = B.rb_batch_solve(b, len(probs), 1e-3, 20000, 50, 16)
        assert nconv == len(probs) and rc == B.RB_OK, (resid, status)
        for i, (A, q, _) in enumerate(probs):
            X = _export(b, i, n[i])
            exact = orc.residual(A, X)
            assert exact <= 3e-3, (i, exact, resid[i])
            assert iters[i] > 0 and status[i] == B.RB_OK
    finally:
        B.rb_batch_destroy(b)


def test_batch_rejects_bad_sizes():
    import torch

    A = to_dev(np.eye(8), torch.float32)
    with pytest.raises(B.RbfgsError):
        B.rb_batch_create([8], [A.data_ptr()], [8], False, [6], 0, stream=stream_ptr())  # q not a multiple of 4
    with pytest.raises(B.RbfgsError):
        B.rb_batch_create([2000], [A.data_ptr()], [2000], False, [8], 0, stream=stream_ptr())  # n > 1024


def test_tile_shapes_give_the_same_iterates():
    # the autotuner's candidates (256 and 512 threads per CTA) sum in the same order, so a batch
    # forced to either shape produces bit-identical iterates; the autotuner picked one of them
    probs = _problems(6, 9)
    b1, n = _create(probs, 13)
    b2, _ = _create(probs, 13)
    try:
        assert B.rb_batch_tile(b1) in (256, 512)
        B.rb_batch_set_tile(b1, 256)
        B.rb_batch_set_tile(b2, 512)
        B.rb_batch_step(b1, 40)
        B.rb_batch_step(b2, 40)
        for i in range(len(probs)):
            assert np.array_equal(_export(b1, i, n[i]), _export(b2, i, n[i])), i
        with pytest.raises(B.RbfgsError):
            B.rb_batch_set_tile(b1, 384)
    finally:
        B.rb_batch_destroy(b1)
        B.rb_batch_destroy(b2)


def test_batch_indefinite_block_fails_only_its_problem():
    # positive diagonal (the trace weights are valid) but the 2 x 2 leading block [[1, 2], [2, 1]] is
    # indefinite: the Cholesky of every block that contains it breaks down, so the first step of that
    # problem reports RB_ENOTSPD and leaves its iterate at X0 = I; the other problem steps normally
    import torch

    n0 = 16
    Abad = np.eye(n0)
    Abad[0, 1] = Abad[1, 0] = 2.0
    Agood, _, _ = wl.spd_spectrum(24, 10.0, 7)
    probs = [(Abad, 4, 0.0), (Agood.astype(np.float32).astype(np.float64), 8, 10.0)]
    b, n = _create(probs, 3)
    try:
        B.rb_batch_step(b, 40)
        rc, iters, resid, status, nconv = B.rb_batch_solve(b, len(probs), 1e-30, 1, 1, 8)
        assert status[0] == B.RB_ENOTSPD and status[1] != B.RB_ENOTSPD, status
        assert np.array_equal(_export(b, 0, n[0]), np.eye(n0, dtype=np.float32))
        _, X = orc.rbfgs_run(probs[1][0], np.eye(n[1]), 8, orc.SKETCH_COORD_TRACE, 3, 1, 0, 41)
        assert rel(_export(b, 1, n[1]), X) <= 1e-4
    finally:
        B.rb_batch_destroy(b)
