"""rbfgs_sigma_noalloc: the power-iteration ||A||_2 estimate for callers that
cannot allocate device memory (a fixed device-memory plan, or an outer
allocator that owns every byte).  Its output must equal what the allocating
path (newton_schulz_init, then rbfgs_sigma) returns for the same matrix, on
two calls in a row (the second call reuses the static scratch the first one
left behind).  This file is collected last on purpose."""
import numpy as np
import pytest

import paper_1602_01768_gb300._binding as B
from paper_1602_01768_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _allocating_sigma(A_dev, n, fp64, iters, stream):
    h = B.newton_schulz_init(n, A_dev.data_ptr(), n, fp64, B.RB_FP64 if fp64 else B.RB_FP32, iters, 0.0, stream)
    try:
        return B.rbfgs_sigma(h)
    finally:
        B.rbfgs_destroy(h)


@pytest.mark.parametrize("fp64", [True, False])
def test_sigma_noalloc_matches_allocating_entry_point(fp64):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    iters = 60
    for n, seed in ((300, 41), (1031, 42)):  # two calls in a row, different sizes
        A, _, lam = wl.spd_spectrum(n, 25.0, seed)
        dt = torch.float64 if fp64 else torch.float32
        Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(device="cuda", dtype=dt)
        ref = _allocating_sigma(Ad, n, fp64, iters, stream)
        got = B.rbfgs_sigma_noalloc(n, Ad.data_ptr(), n, fp64, iters, stream)
        tol = 1e-12 if fp64 else 1e-6
        assert abs(got - ref) <= tol * ref, (n, got, ref)
        assert abs(got - lam.max()) <= 0.05 * lam.max()


def test_sigma_noalloc_rejects_oversize():
    with pytest.raises(B.RbfgsError) as e:
        B.rbfgs_sigma_noalloc(65537, 1, 65537, True, 1, 0)
    assert e.value.status == B.RB_EINVAL
