"""Seeded synthetic SPD inputs shaped like the paper's test matrices.

This module holds no arithmetic of the method: it only builds input matrices
(and the arrival stream of the serving workload).  Both the CUDA path and the
CPU oracle receive the SAME matrices from here.

The paper's own inputs (Sec. 10: LIBSVM ridge Hessians, UF sparse matrices,
MATLAB ``rand`` Gram matrices) are not available offline; the generators below
stand in for them with the same structure:

* ``spd_spectrum``   A = U diag(lam) U^T, U Haar-orthogonal (QR of a Gaussian
  with the sign of diag(R) fixed), lam log-uniform in [lam_max/kappa, lam_max].
* ``spd_gram``       A = M^T M / m + shift I (ridge-Hessian form of Sec. 10.2),
  M Gaussian, optionally with log-uniform column scales or at a given density.
* ``spd_uniform_gram``  A = Abar^T Abar, Abar uniform [0,1] (Sec. 10.1).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian, columns signed by diag(R)."""
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def spd_spectrum(n: int, kappa: float, seed: int, lam_max: float = 1.0):
    """A = U diag(lam) U^T with lam log-uniform in [lam_max/kappa, lam_max].

    The extreme eigenvalues are placed exactly at the ends so that kappa(A)
    equals ``kappa``.  Returns (A, U, lam) in float64, A in Fortran order.
    """
    rng = _rng(seed)
    U = haar_orthogonal(n, rng)
    lo = math.log(lam_max / kappa)
    hi = math.log(lam_max)
    lam = np.exp(rng.uniform(lo, hi, size=n))
    if n >= 2:
        lam[0] = lam_max / kappa
        lam[1] = lam_max
    A = (U * lam[None, :]) @ U.T
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A), U, lam


def spd_gram(n: int, m: int, shift: float, seed: int, col_scale_range=None,
             density: float = 1.0, dtype=np.float64):
    """A = M^T M / m + shift I with M (m x n) i.i.d. N(0,1) (CPU, numpy).

    ``col_scale_range=(a, b)`` multiplies column j of M by a log-uniform factor
    in [a, b]; ``density < 1`` keeps each entry with that probability.
    """
    rng = _rng(seed)
    M = rng.standard_normal((m, n))
    if density < 1.0:
        M *= rng.random((m, n)) < density
    if col_scale_range is not None:
        a, b = col_scale_range
        M *= np.exp(rng.uniform(math.log(a), math.log(b), size=n))[None, :]
    A = (M.T @ M) / m
    A[np.diag_indices(n)] += shift
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A.astype(dtype))


def spd_gram_torch(n: int, m: int, shift: float, seed: int, device, col_scale_range=None,
                   density: float = 1.0, chunk: int = 8192):
    """Same construction as ``spd_gram`` on a torch device, FP32 result.

    Used for the n = 16384 workload (M is 65536 x 16384), where a CPU build
    would take minutes.  M is generated and accumulated in row chunks of
    ``chunk`` so the device never holds all of M.  The product is taken in
    FP32 with TF32 disabled; the result is an input matrix, not a quantity
    under test.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    prev = torch.backends.cuda.matmul.allow_tf32 if torch.cuda.is_available() else None
    if prev is not None:
        torch.backends.cuda.matmul.allow_tf32 = False
    try:
        scale = None
        if col_scale_range is not None:
            a, b = col_scale_range
            u = torch.rand(n, generator=g, device=device, dtype=torch.float32)
            scale = torch.exp(math.log(a) + u * (math.log(b) - math.log(a)))
        A = torch.zeros(n, n, device=device, dtype=torch.float32)
        done = 0
        while done < m:
            r = min(chunk, m - done)
            Mc = torch.randn(r, n, generator=g, device=device, dtype=torch.float32)
            if density < 1.0:
                keep = torch.rand(r, n, generator=g, device=device, dtype=torch.float32) < density
                Mc = Mc * keep
            if scale is not None:
                Mc = Mc * scale[None, :]
            A.addmm_(Mc.t(), Mc)
            done += r
            del Mc
        A.div_(m)
        A.diagonal().add_(shift)
        A = 0.5 * (A + A.t())
        return A.contiguous()
    finally:
        if prev is not None:
            torch.backends.cuda.matmul.allow_tf32 = prev


def spd_uniform_gram(n: int, seed: int):
    """A = Abar^T Abar with Abar uniform on [0,1]^{n x n} (Sec. 10.1 synthetic)."""
    rng = _rng(seed)
    B = rng.random((n, n))
    A = B.T @ B
    return np.asfortranarray(0.5 * (A + A.T))


def spd_uniform_gram_torch(n: int, seed: int, device):
    """Same construction as ``spd_uniform_gram`` on a torch device, FP32 (TF32 off): the large
    sizes of Sec. 10.1, where a CPU build would take hours."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        Bm = torch.rand(n, n, generator=g, device=device, dtype=torch.float32)
        A = Bm.t() @ Bm
        del Bm
        A = 0.5 * (A + A.t())
        return A.contiguous()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


# --------------------------------------------------------------------------
# The five workloads (sizes, spectra and sketch choices).
# --------------------------------------------------------------------------
WORKLOADS = {
    "c1_rbfgs_fp64_n256": dict(n=256, q=8, kappa=1e2, method="rbfgs", sketch="gauss",
                               prec="fp64", max_iter=300, tol=1e-8, seed=1),
    "c2_adarbfgs_n4096": dict(n=4096, q=64, m=16384, shift=1e-3, col_scale=(1e-2, 1.0),
                              method="adarbfgs", sketch="gauss", tol=1e-4, seed=2),
    "c3_adarbfgs_n16384": dict(n=16384, q=128, m=65536, shift=1e-4, density=0.01,
                               method="adarbfgs", sketch="gauss", tol=1e-4, seed=3),
    "c4_batched_coord": dict(count=512, n_range=(32, 1024), kappa_range=(1e1, 1e4),
                             q_choices=(4, 8, 16, 32), method="rbfgs", sketch="coord_trace",
                             tol=1e-5, seed=4),
    "c5_serving": dict(requests=4000, rate=200.0, n_range=(512, 8192), m_factor=2,
                       shift=1e-3, tols=(1e-3, 1e-4, 1e-6), budget_bytes=120 * 2**30, seed=5),
}


def c1_matrix():
    w = WORKLOADS["c1_rbfgs_fp64_n256"]
    return spd_spectrum(w["n"], w["kappa"], w["seed"])


def c2_matrix(n: int | None = None, m: int | None = None, device=None):
    """c2: A = M^T M/m + 1e-3 I, M Gaussian with column scales log-uniform in [1e-2, 1].

    ``n``/``m`` shrink the same recipe for tests (m = 4 n keeps the spectrum shape).
    """
    w = WORKLOADS["c2_adarbfgs_n4096"]
    n = n or w["n"]
    m = m or (w["m"] * n) // w["n"]
    if device is not None:
        return spd_gram_torch(n, m, w["shift"], w["seed"], device, col_scale_range=w["col_scale"])
    return spd_gram(n, m, w["shift"], w["seed"], col_scale_range=w["col_scale"])


def c3_matrix(n: int | None = None, device=None):
    """c3: A = M^T M/m + 1e-4 I, M (4n x n) 1%-dense N(0,1), FP32 on ``device``."""
    w = WORKLOADS["c3_adarbfgs_n16384"]
    n = n or w["n"]
    m = 4 * n
    if device is not None:
        return spd_gram_torch(n, m, w["shift"], w["seed"], device, density=w["density"])
    return spd_gram(n, m, w["shift"], w["seed"], density=w["density"])


def c4_problems(count: int | None = None, seed: int | None = None):
    """c4: list of (A, q, kappa) with n log-uniform in [32, 1024], kappa log-uniform
    in [1e1, 1e4], q uniform in {4, 8, 16, 32}."""
    w = WORKLOADS["c4_batched_coord"]
    count = count or w["count"]
    rng = _rng(seed if seed is not None else w["seed"])
    lo, hi = w["n_range"]
    klo, khi = w["kappa_range"]
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        kappa = float(math.exp(rng.uniform(math.log(klo), math.log(khi))))
        q = int(rng.choice(w["q_choices"]))
        A, _, _ = spd_spectrum(n, kappa, 1000 + i + 100000 * (seed or 0))
        out.append((A, q, kappa))
    return out


def c5_stream(requests: int | None = None, rate: float | None = None, seed: int | None = None):
    """c5: Poisson arrivals; each request (t_arrival, n, tol, q, seed).  q = 32 round(sqrt(n)/32), >= 32."""
    w = WORKLOADS["c5_serving"]
    requests = requests or w["requests"]
    rate = rate or w["rate"]
    rng = _rng(seed if seed is not None else w["seed"])
    lo, hi = w["n_range"]
    t = 0.0
    out = []
    for i in range(requests):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        tol = float(rng.choice(w["tols"]))
        q = max(32, 32 * int(round(math.sqrt(n) / 32)))
        out.append(dict(t=t, n=n, tol=tol, q=q, seed=10_000 + i))
    return out


def c5_matrix(n: int, seed: int, device=None):
    w = WORKLOADS["c5_serving"]
    if device is not None:
        return spd_gram_torch(n, w["m_factor"] * n, w["shift"], seed, device)
    return spd_gram(n, w["m_factor"] * n, w["shift"], seed)
