"""ctypes front end of the FP64 CPU oracle (oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never
imports this module.  All arrays are float64, Fortran (column-major) order.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

TAG_COORD = 0xC0000000
TAG_COLS = 0xD0000000

SKETCH_GAUSS = 0
SKETCH_COORD_TRACE = 1
SKETCH_COORD_UNIFORM = 2


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i, u32, u64, p = C.c_double, C.c_int, C.c_uint32, C.c_uint64, C.c_void_p
        sig = {
            "orc_philox4x32_10": (None, [p, p, p]),
            "orc_gauss_sketch": (None, [u64, u64, u64, i, i, p]),
            "orc_floyd_sample": (None, [u64, u64, u64, u32, i, i, p]),
            "orc_coord_trace_block": (i, [p, i, i, u64, u64, u64, p, p]),
            "orc_cholesky": (i, [i, p]),
            "orc_gauss_jordan": (i, [i, p, p]),
            "orc_rbfgs_step": (i, [i, p, p, p, i, i]),
            "orc_adarbfgs_step": (i, [i, p, p, p, i]),
            "orc_rbfgs_run": (i, [i, p, p, i, i, u64, u64, u64, i, i]),
            "orc_adarbfgs_run": (i, [i, p, p, i, i, u64, u64, u64, i]),
            "orc_aip_step": (i, [i, p, p, p, i]),
            "orc_aip_run": (i, [i, p, p, i, i, u64, u64, u64, i]),
            "orc_ns_step": (None, [i, p, p]),
            "orc_power_norm": (d, [i, p, i]),
            "orc_ns_init": (None, [i, p, d, p]),
            "orc_mr_step": (d, [i, p, p]),
            "orc_mr_init": (None, [i, p, p]),
            "orc_residual": (d, [i, p, p]),
            "orc_residual_factored": (d, [i, p, p]),
            "orc_residual_sampled": (d, [i, p, p, p, i, u64]),
            "orc_logf32": (C.c_float, [C.c_float]),
            "orc_sincospif32": (None, [C.c_float, p, p]),
            "orc_round_tf32": (C.c_float, [C.c_float]),
            "orc_set_threads": (None, [i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _f64(a):
    a = np.asarray(a, dtype=np.float64)
    return np.asfortranarray(a)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def logf32(u):
    """The sketch generator's binary32 natural log (oracle.c, orc_logf32)."""
    return np.float32(lib().orc_logf32(float(np.float32(u))))


def sincospif32(x):
    """The sketch generator's binary32 (sin(pi x), cos(pi x)) (orc_sincospif32)."""
    s, c = C.c_float(), C.c_float()
    lib().orc_sincospif32(float(np.float32(x)), C.byref(s), C.byref(c))
    return np.float32(s.value), np.float32(c.value)


def round_tf32(z):
    return np.float32(lib().orc_round_tf32(float(np.float32(z))))


def gauss_sketch(seed, stream, k, n, q):
    S = np.zeros((n, q), dtype=np.float64, order="F")
    lib().orc_gauss_sketch(seed, stream, k, n, q, _ptr(S))
    return S


def floyd_sample(seed, stream, k, tag, n, m):
    out = np.zeros(m, dtype=np.int32)
    lib().orc_floyd_sample(seed, stream, k, tag, n, m, _ptr(out))
    return out


def coord_trace_block(A, q, seed, stream, k):
    A = _f64(A)
    first = np.zeros(1, dtype=np.int32)
    size = np.zeros(1, dtype=np.int32)
    b = lib().orc_coord_trace_block(_ptr(A), A.shape[0], q, seed, stream, k, _ptr(first), _ptr(size))
    return b, int(first[0]), int(size[0])


def cholesky(M):
    M = _f64(M).copy(order="F")
    rc = lib().orc_cholesky(M.shape[0], _ptr(M))
    return rc, M


def gauss_jordan(A):
    A = _f64(A)
    out = np.zeros_like(A, order="F")
    rc = lib().orc_gauss_jordan(A.shape[0], _ptr(A), _ptr(out))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def rbfgs_step(A, X, S, form=1):
    A, S = _f64(A), _f64(S)
    X = _f64(X).copy(order="F")
    rc = lib().orc_rbfgs_step(A.shape[0], _ptr(A), _ptr(X), _ptr(S), S.shape[1], form)
    return rc, X


def adarbfgs_step(A, L, St):
    A, St = _f64(A), _f64(St)
    L = _f64(L).copy(order="F")
    rc = lib().orc_adarbfgs_step(A.shape[0], _ptr(A), _ptr(L), _ptr(St), St.shape[1])
    return rc, L


def rbfgs_run(A, X0, q, kind, seed, stream, k0, nsteps, form=1):
    A = _f64(A)
    X = _f64(X0).copy(order="F")
    done = lib().orc_rbfgs_run(A.shape[0], _ptr(A), _ptr(X), q, kind, seed, stream, k0, nsteps, form)
    return done, X


def adarbfgs_run(A, L0, q, kind, seed, stream, k0, nsteps):
    A = _f64(A)
    L = _f64(L0).copy(order="F")
    done = lib().orc_adarbfgs_run(A.shape[0], _ptr(A), _ptr(L), q, kind, seed, stream, k0, nsteps)
    return done, L


def aip_step(A, X, S):
    """One step of Eq. (BFGSas): X+ = X + S (S^T A S)^-1 S^T (I - A X)."""
    A, S = _f64(A), _f64(S)
    X = _f64(X).copy(order="F")
    rc = lib().orc_aip_step(A.shape[0], _ptr(A), _ptr(X), _ptr(S), S.shape[1])
    return rc, X


def aip_run(A, X0, q, kind, seed, stream, k0, nsteps):
    A = _f64(A)
    X = _f64(X0).copy(order="F")
    done = lib().orc_aip_run(A.shape[0], _ptr(A), _ptr(X), q, kind, seed, stream, k0, nsteps)
    return done, X


def ns_step(A, X):
    A = _f64(A)
    X = _f64(X).copy(order="F")
    lib().orc_ns_step(A.shape[0], _ptr(A), _ptr(X))
    return X


def power_norm(A, iters):
    A = _f64(A)
    return lib().orc_power_norm(A.shape[0], _ptr(A), iters)


def ns_init(A, sigma):
    A = _f64(A)
    X = np.zeros_like(A, order="F")
    lib().orc_ns_init(A.shape[0], _ptr(A), sigma, _ptr(X))
    return X


def mr_step(A, X):
    A = _f64(A)
    X = _f64(X).copy(order="F")
    alpha = lib().orc_mr_step(A.shape[0], _ptr(A), _ptr(X))
    return alpha, X


def mr_init(A):
    A = _f64(A)
    X = np.zeros_like(A, order="F")
    lib().orc_mr_init(A.shape[0], _ptr(A), _ptr(X))
    return X


def residual(A, X):
    A, X = _f64(A), _f64(X)
    return lib().orc_residual(A.shape[0], _ptr(A), _ptr(X))


def residual_factored(A, L):
    A, L = _f64(A), _f64(L)
    return lib().orc_residual_factored(A.shape[0], _ptr(A), _ptr(L))


def residual_sampled(A, m, col_seed, X=None, L=None):
    A = _f64(A)
    Xc = _f64(X) if X is not None else None
    Lc = _f64(L) if L is not None else None
    Xp = _ptr(Xc) if Xc is not None else None
    Lp = _ptr(Lc) if Lc is not None else None
    return lib().orc_residual_sampled(A.shape[0], _ptr(A), Xp, Lp, m, col_seed)


def set_threads(threads):
    """Threads of the oracle's OpenMP loops from now on."""
    lib().orc_set_threads(int(threads))


def n_threads():
    """Threads the OpenMP runtime of the oracle uses (OMP_NUM_THREADS or all cores)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env:
        return int(env)
    return len(os.sched_getaffinity(0))
