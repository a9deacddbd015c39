"""ctypes binding of include/rbfgs.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of its own.  Device buffers are passed as raw pointers (for
example ``tensor.data_ptr()``); streams as ``cudaStream_t`` integers.  A
failing status raises :class:`RbfgsError`; ``RB_NOTCONV`` is returned.
"""
import ctypes as C
import os

from . import build as _build

RB_OK, RB_NOTCONV = 0, 1
RB_EINVAL, RB_ENOMEM, RB_ECUDA, RB_ENOTSPD, RB_ENONFINITE, RB_ETIMEOUT, RB_EUNSUPPORTED = -1, -2, -3, -4, -5, -6, -7

RB_FP64, RB_FP32, RB_TF32, RB_TF32X3, RB_MIXED, RB_BF16, RB_BF16X3 = 0, 1, 2, 3, 4, 5, 6
RB_SKETCH_GAUSS, RB_SKETCH_COORD_TRACE, RB_SKETCH_COORD_UNIFORM = 0, 1, 2
RB_METHOD_RBFGS, RB_METHOD_ADARBFGS, RB_METHOD_NS, RB_METHOD_MR, RB_METHOD_AIP = 0, 1, 2, 3, 4
RB_WHAT_X, RB_WHAT_L = 0, 1

PREC = {"fp64": RB_FP64, "fp32": RB_FP32, "tf32": RB_TF32, "tf32x3": RB_TF32X3, "mixed": RB_MIXED, "bf16": RB_BF16,
        "bf16x3": RB_BF16X3}


class RbOpts(C.Structure):
    _fields_ = [("method", C.c_int32), ("sketch", C.c_int32), ("q", C.c_int32), ("prec", C.c_int32),
                ("seed", C.c_uint64), ("stream_id", C.c_uint64), ("power_iters", C.c_int32),
                ("core_fp64", C.c_int32), ("reserved", C.c_int32 * 6)]


class RbfgsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib().rbfgs_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


_LIB = None

# name -> (restype, argtypes)
_SIGS = {
    "rbfgs_default_opts": (None, [C.c_void_p]),
    "rbfgs_status_string": (C.c_char_p, [C.c_int]),
    "rbfgs_init": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "rbfgs_step": (C.c_int, [C.c_void_p, C.c_int]),
    "aip_step": (C.c_int, [C.c_void_p, C.c_int]),
    "adarbfgs_step": (C.c_int, [C.c_void_p, C.c_int]),
    "rbfgs_residual": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_void_p]),
    "rbfgs_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                              C.c_void_p]),
    "rbfgs_export": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "rbfgs_import": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "rbfgs_set_step": (C.c_int, [C.c_void_p, C.c_uint64]),
    "rbfgs_get_step": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rbfgs_sync": (C.c_int, [C.c_void_p]),
    "rbfgs_draw_sketch": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64]),
    "newton_schulz_init": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                                     C.c_double, C.c_void_p]),
    "newton_schulz_step": (C.c_int, [C.c_void_p, C.c_int]),
    "mr_init": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p]),
    "mr_step": (C.c_int, [C.c_void_p, C.c_int]),
    "rbfgs_sigma": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rbfgs_core64": (C.c_int, [C.c_int, C.c_void_p, C.c_float, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "rbfgs_sigma_noalloc": (C.c_int, [C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "rbfgs_load_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "rbfgs_export_host": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "rbfgs_profile_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "rbfgs_launch_count": (C.c_int, [C.c_void_p]),
    "rbfgs_wait_selftest": (C.c_int, [C.c_void_p, C.c_int64]),
    "rbfgs_reset": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64]),
    "rbfgs_destroy": (C.c_int, [C.c_void_p]),
    "rb_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_uint64, C.c_void_p]),
    "rb_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "rb_batch_residual": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_void_p]),
    "rb_batch_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "rb_batch_export": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "rb_batch_destroy": (C.c_int, [C.c_void_p]),
    "rb_batch_tile": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rb_batch_set_tile": (C.c_int, [C.c_void_p, C.c_int]),
    "rbfgs_residual_start": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64]),
    "rbfgs_residual_poll": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbfgs_footprint": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p]),
    "rb_next_check_gap": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double]),
    "rb_srv_create": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "rb_srv_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_double,
                                C.c_uint64, C.c_int, C.c_void_p, C.c_int, C.c_int64, C.c_void_p]),
    "rb_srv_poll": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "rb_srv_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p]),
    "rb_srv_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rb_srv_destroy": (C.c_int, [C.c_void_p]),
}


def library_path():
    return _build.LIB


def _lib():
    """Load the sm_103a library (building it in-tree first if it is missing).

    There is no fallback: if the library cannot be built or loaded, this
    raises, and nothing of the method runs.
    """
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            _build.build()
        L = C.CDLL(path, mode=C.RTLD_GLOBAL)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIGS.keys())


def _check(st, where):
    if st < 0:
        raise RbfgsError(st, where)
    return st


def _p(x):
    return None if x is None else C.c_void_p(int(x))


def rbfgs_status_string(status):
    return _lib().rbfgs_status_string(status).decode()


def rbfgs_default_opts():
    o = RbOpts()
    _lib().rbfgs_default_opts(C.byref(o))
    return o


def make_opts(method=RB_METHOD_RBFGS, sketch=RB_SKETCH_GAUSS, q=8, prec=RB_FP64, seed=0, stream_id=0,
              power_iters=0, core_fp64=0):
    o = rbfgs_default_opts()
    o.method, o.sketch, o.q, o.prec = method, sketch, q, prec
    o.seed, o.stream_id, o.power_iters, o.core_fp64 = seed, stream_id, power_iters, int(core_fp64)
    return o


def rbfgs_init(n, A_dev, lda, a_is_fp64, opts, stream=0):
    h = C.c_void_p()
    _check(_lib().rbfgs_init(C.byref(h), n, _p(A_dev), lda, int(a_is_fp64), C.byref(opts), _p(stream)),
           "rbfgs_init")
    return h


def rbfgs_step(h, nsteps):
    return _check(_lib().rbfgs_step(h, nsteps), "rbfgs_step")


def aip_step(h, nsteps):
    return _check(_lib().aip_step(h, nsteps), "aip_step")


def adarbfgs_step(h, nsteps):
    return _check(_lib().adarbfgs_step(h, nsteps), "adarbfgs_step")


def rbfgs_residual(h, ncols=0, col_seed=0):
    out = C.c_double()
    _check(_lib().rbfgs_residual(h, ncols, col_seed, C.byref(out)), "rbfgs_residual")
    return out.value


def rbfgs_solve(h, tol, max_iter, check_every, check_cols, confirm_cols):
    it = C.c_int()
    r = C.c_double()
    st = _check(_lib().rbfgs_solve(h, tol, max_iter, check_every, check_cols, confirm_cols, C.byref(it),
                                   C.byref(r)), "rbfgs_solve")
    return st, it.value, r.value


def rb_next_check_gap(e, k0, r0, k1, r1, tol):
    return int(_lib().rb_next_check_gap(e, k0, r0, k1, r1, tol))


def rbfgs_export(h, what, out_dev, ld):
    return _check(_lib().rbfgs_export(h, what, _p(out_dev), ld), "rbfgs_export")


def rbfgs_import(h, what, in_dev, ld):
    return _check(_lib().rbfgs_import(h, what, _p(in_dev), ld), "rbfgs_import")


def rbfgs_set_step(h, k):
    return _check(_lib().rbfgs_set_step(h, k), "rbfgs_set_step")


def rbfgs_get_step(h):
    k = C.c_uint64()
    _check(_lib().rbfgs_get_step(h, C.byref(k)), "rbfgs_get_step")
    return k.value


def rbfgs_draw_sketch(h, k, out_dev, ld):
    return _check(_lib().rbfgs_draw_sketch(h, k, _p(out_dev), ld), "rbfgs_draw_sketch")


def rbfgs_sync(h):
    return _check(_lib().rbfgs_sync(h), "rbfgs_sync")


def newton_schulz_init(n, A_dev, lda, a_is_fp64, prec, power_iters=0, sigma_override=0.0, stream=0):
    h = C.c_void_p()
    _check(_lib().newton_schulz_init(C.byref(h), n, _p(A_dev), lda, int(a_is_fp64), prec, power_iters,
                                     sigma_override, _p(stream)), "newton_schulz_init")
    return h


def newton_schulz_step(h, nsteps):
    return _check(_lib().newton_schulz_step(h, nsteps), "newton_schulz_step")


def mr_init(n, A_dev, lda, a_is_fp64, prec, stream=0):
    h = C.c_void_p()
    _check(_lib().mr_init(C.byref(h), n, _p(A_dev), lda, int(a_is_fp64), prec, _p(stream)), "mr_init")
    return h


def mr_step(h, nsteps):
    return _check(_lib().mr_step(h, nsteps), "mr_step")


def rbfgs_sigma(h):
    s = C.c_double()
    _check(_lib().rbfgs_sigma(h, C.byref(s)), "rbfgs_sigma")
    return s.value


def rbfgs_core64(q, M_dev, s, out_dev, ldo, cluster=1, stream=0):
    """Returns the CTAs that ran."""
    c = C.c_int(cluster)
    _check(_lib().rbfgs_core64(q, _p(M_dev), s, _p(out_dev), ldo, C.byref(c), _p(stream)), "rbfgs_core64")
    return c.value


def rbfgs_sigma_noalloc(n, A_dev, lda, a_is_fp64, power_iters=0, stream=0):
    s = C.c_double()
    _check(_lib().rbfgs_sigma_noalloc(n, _p(A_dev), lda, int(a_is_fp64), power_iters, C.byref(s), _p(stream)),
           "rbfgs_sigma_noalloc")
    return s.value


def rbfgs_load_host(h, A_host, lda, a_is_fp64):
    return _check(_lib().rbfgs_load_host(h, _p(A_host), lda, int(a_is_fp64)), "rbfgs_load_host")


def rbfgs_export_host(h, what, out_host, ld):
    return _check(_lib().rbfgs_export_host(h, what, _p(out_host), ld), "rbfgs_export_host")


def rbfgs_profile_step(h, cap=24):
    ms = (C.c_double * cap)()
    names = (C.c_char_p * cap)()
    n = C.c_int()
    _check(_lib().rbfgs_profile_step(h, ms, names, cap, C.byref(n)), "rbfgs_profile_step")
    return [(names[i].decode(), ms[i]) for i in range(n.value)]


def rbfgs_reset(h, seed, stream_id=0):
    return _check(_lib().rbfgs_reset(h, seed, stream_id), "rbfgs_reset")


def rbfgs_wait_selftest(h, limit_cycles):
    return _check(_lib().rbfgs_wait_selftest(h, int(limit_cycles)), "rbfgs_wait_selftest")


def rbfgs_launch_count():
    c = C.c_uint64()
    _check(_lib().rbfgs_launch_count(C.byref(c)), "rbfgs_launch_count")
    return c.value


def rbfgs_destroy(h):
    return _check(_lib().rbfgs_destroy(h), "rbfgs_destroy")


def rb_batch_create(n_list, A_ptrs, lda_list, a_is_fp64, q_list, seed, stream_ids=None, stream=0):
    cnt = len(n_list)
    n_arr = (C.c_int * cnt)(*n_list)
    q_arr = (C.c_int * cnt)(*q_list)
    a_arr = (C.c_void_p * cnt)(*[int(p) for p in A_ptrs])
    l_arr = (C.c_int64 * cnt)(*lda_list)
    s_arr = (C.c_uint64 * cnt)(*stream_ids) if stream_ids is not None else None
    b = C.c_void_p()
    _check(_lib().rb_batch_create(C.byref(b), cnt, n_arr, a_arr, l_arr, int(a_is_fp64), q_arr,
                                  s_arr, seed, _p(stream)), "rb_batch_create")
    b._count = cnt
    return b


def rb_batch_step(b, steps):
    return _check(_lib().rb_batch_step(b, steps), "rb_batch_step")


def rb_batch_residual(b, count, ncols, col_seed):
    out = (C.c_double * count)()
    _check(_lib().rb_batch_residual(b, ncols, col_seed, out), "rb_batch_residual")
    return list(out)


def rb_batch_solve(b, count, tol, max_iter, check_every, ncols):
    it = (C.c_int * count)()
    r = (C.c_double * count)()
    st = (C.c_int * count)()
    nc = C.c_int()
    rc = _check(_lib().rb_batch_solve(b, tol, max_iter, check_every, ncols, it, r, st, C.byref(nc)),
                "rb_batch_solve")
    return rc, list(it), list(r), list(st), nc.value


def rb_batch_export(b, i, out_dev, ld):
    return _check(_lib().rb_batch_export(b, i, _p(out_dev), ld), "rb_batch_export")


def rb_batch_tile(b):
    t = C.c_int()
    _check(_lib().rb_batch_tile(b, C.byref(t)), "rb_batch_tile")
    return t.value


def rb_batch_set_tile(b, threads_per_cta):
    return _check(_lib().rb_batch_set_tile(b, threads_per_cta), "rb_batch_set_tile")


def rb_batch_destroy(b):
    return _check(_lib().rb_batch_destroy(b), "rb_batch_destroy")


def rbfgs_residual_start(h, ncols, col_seed):
    return _check(_lib().rbfgs_residual_start(h, ncols, col_seed), "rbfgs_residual_start")


def rbfgs_residual_poll(h):
    ready = C.c_int()
    out = C.c_double()
    _check(_lib().rbfgs_residual_poll(h, C.byref(ready), C.byref(out)), "rbfgs_residual_poll")
    return bool(ready.value), out.value


def rbfgs_footprint(n, opts):
    b = C.c_size_t()
    _check(_lib().rbfgs_footprint(n, C.byref(opts), C.byref(b)), "rbfgs_footprint")
    return b.value


class SrvResult(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("status", C.c_int32), ("iters", C.c_int32), ("resid", C.c_double),
                ("latency_s", C.c_double), ("queue_s", C.c_double), ("n", C.c_int32), ("q", C.c_int32),
                ("prec", C.c_int32), ("floor_limited", C.c_int32)]


class SrvStats(C.Structure):
    _fields_ = [("completed", C.c_int32), ("failed", C.c_int32), ("queued", C.c_int32), ("live", C.c_int32),
                ("p50_s", C.c_double), ("p99_s", C.c_double), ("solves_per_s", C.c_double),
                ("hbm_in_use", C.c_uint64)]


def rb_srv_create(hbm_budget_bytes, max_live, prec=RB_MIXED, check_every=32, check_cols=256, max_iter=20000):
    s = C.c_void_p()
    _check(_lib().rb_srv_create(C.byref(s), hbm_budget_bytes, max_live, prec, check_every, check_cols, max_iter),
           "rb_srv_create")
    return s


def rb_srv_submit(s, n, A, a_on_device, lda, a_is_fp64, tol, seed, q=0, out=None, out_on_device=False, ldo=0):
    t = C.c_int64()
    _check(_lib().rb_srv_submit(s, n, _p(A), int(a_on_device), lda, int(a_is_fp64), tol, seed, q, _p(out),
                                int(out_on_device), ldo, C.byref(t)), "rb_srv_submit")
    return t.value


def rb_srv_poll(s, ticket):
    d = C.c_int()
    _check(_lib().rb_srv_poll(s, ticket, C.byref(d)), "rb_srv_poll")
    return bool(d.value)


def rb_srv_wait(s, ticket, timeout_s=600.0):
    r = SrvResult()
    _check(_lib().rb_srv_wait(s, ticket, timeout_s, C.byref(r)), "rb_srv_wait")
    return r


def rb_srv_stats(s):
    st = SrvStats()
    _check(_lib().rb_srv_stats(s, C.byref(st)), "rb_srv_stats")
    return st


def rb_srv_destroy(s):
    return _check(_lib().rb_srv_destroy(s), "rb_srv_destroy")
