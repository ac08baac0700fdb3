"""ctypes binding of the C ABI in include/rte.h (argument marshalling only).

Every function keeps the C name.  Device pointers are passed as integers
(e.g. ``tensor.data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream``
integers.  A non-OK status raises :class:`RteError`, except RTE_ENOCONV from
the solvers, which is reported in the returned stats.

The library must have been built (``paper_1802_03061_gb300.build.build()``);
there is no fallback of any kind when it is missing.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librte.so")

RTE_OK, RTE_EINVAL, RTE_EUNSUPPORTED, RTE_ENOMEM, RTE_ECUDA, RTE_ENOCONV, RTE_ETIMEOUT, RTE_ENAN = range(8)
PREC = {"fp64": 0, "mixed_fp32": 1, "mixed_bf16": 2}


class RteError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s: %s%s" % (where, _status_str(status), (" (%s)" % detail) if detail else ""))


class rte_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3)]


class rte_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("tol", ctypes.c_double), ("restart", ctypes.c_int),
                ("maxit", ctypes.c_int), ("inner_tol", ctypes.c_double), ("use_guess", ctypes.c_int),
                ("q_policy", ctypes.c_int), ("inner_solver", ctypes.c_int), ("precond", ctypes.c_int),
                ("precond_lmax", ctypes.c_int), ("mode_mix", ctypes.c_int)]


class rte_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres_true", ctypes.c_double), ("ms_total", ctypes.c_double), ("ms_pre", ctypes.c_double),
                ("est_err_bound", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rte_instance_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("h", ctypes.c_double), ("mu_t", ctypes.c_double), ("mu_s", ctypes.c_double),
                ("L", ctypes.c_int), ("sigma_hat", ctypes.POINTER(ctypes.c_double)), ("q", ctypes.c_int),
                ("rows_per_block", ctypes.c_int)]


_lib = None
VP = ctypes.c_void_p


def lib():
    """Load librte.so; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librte.so is not built (%s); run paper_1802_03061_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.rte_plan_create.argtypes = [ctypes.POINTER(VP), rte_grid, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(rte_opts), VP]
        for name in ("rte_apply_K", "rte_apply_A", "rte_apply_K32", "rte_apply_K64e", "rte_apply_precond32", "rte_rhs"):
            getattr(L, name).argtypes = [VP, VP, VP, VP]
        L.rte_solve.argtypes = [VP, VP, VP, ctypes.POINTER(rte_opts), ctypes.POINTER(rte_stats), VP]
        L.rte_solve_host.argtypes = [VP, VP, VP, ctypes.POINTER(rte_opts), ctypes.POINTER(rte_stats), VP]
        L.rte_plan_info.argtypes = [VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)]
        L.rte_plan_cell_weights.argtypes = [VP, ctypes.POINTER(ctypes.c_double)]
        L.rte_precond_info.argtypes = [VP, ctypes.POINTER(ctypes.c_int)]
        L.rte_inhom_create.argtypes = [ctypes.POINTER(VP), ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_double), VP]
        L.rte_inhom_apply32.argtypes = [VP, VP, VP, VP]
        L.rte_inhom_apply64.argtypes = [VP, VP, VP, VP]
        L.rte_inhom_diag.argtypes = [VP, ctypes.POINTER(ctypes.c_double)]
        L.rte_inhom_destroy.argtypes = [VP]
        L.rte_aniso3d_create.argtypes = [ctypes.POINTER(VP), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double), VP]
        L.rte_aniso3d_info.argtypes = [VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.rte_aniso3d_pair_table.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.rte_aniso3d_cell_weights.argtypes = [VP, ctypes.POINTER(ctypes.c_double)]
        for name in ("rte_aniso3d_apply_K", "rte_aniso3d_apply_K64e", "rte_aniso3d_apply_K32", "rte_aniso3d_rhs"):
            getattr(L, name).argtypes = [VP, VP, VP, VP]
        L.rte_aniso3d_solve.argtypes = [VP, VP, VP, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(rte_stats), VP]
        L.rte_aniso3d_destroy.argtypes = [VP]
        L.rte_destroy.argtypes = [VP]
        L.rte_time_passes.argtypes = [VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), VP]
        L.rte_time_passes.restype = ctypes.c_int
        L.rte_kernel_launches.restype = ctypes.c_longlong
        L.rte_debug_fail_alloc.argtypes = [ctypes.c_long, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                           ctypes.POINTER(ctypes.c_long)]
        L.rte_debug_fail_alloc.restype = ctypes.c_int
        L.rte_apply_K_noalloc.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_double), VP, VP, VP]
        L.rte_apply_K_noalloc.restype = ctypes.c_int
        L.rte_noalloc_scratch_bytes.restype = ctypes.c_longlong
        L.rte_batch_create.argtypes = [ctypes.POINTER(VP), ctypes.c_int, ctypes.POINTER(rte_instance_desc),
                                       ctypes.POINTER(rte_opts), VP]
        L.rte_batch_layout.argtypes = [VP, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]
        L.rte_batch_solve.argtypes = [VP, ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(rte_stats), VP]
        L.rte_batch_solve_packed.argtypes = [VP, VP, VP, ctypes.POINTER(rte_stats), ctypes.POINTER(ctypes.c_double),
                                             VP]
        L.rte_batch_destroy.argtypes = [VP]
        L.rte_autotune.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), VP]
        for name in ("rte_batch_create", "rte_batch_layout", "rte_batch_solve", "rte_batch_solve_packed",
                     "rte_batch_destroy", "rte_autotune"):
            getattr(L, name).restype = ctypes.c_int
        FP = ctypes.POINTER(ctypes.c_float)
        L.rte_cnn_create.argtypes = [ctypes.POINTER(VP), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_ulonglong, VP]
        L.rte_cnn_destroy.argtypes = [VP]
        L.rte_cnn_forward.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, VP, VP]
        L.rte_cnn_train_step.argtypes = [VP, VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_float, FP, VP]
        L.rte_cnn_layer.argtypes = [VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(VP)]
        L.rte_cnn_sync_weights.argtypes = [VP, VP]
        L.rte_cnn_save.argtypes = [VP, ctypes.c_char_p]
        L.rte_cnn_load.argtypes = [VP, ctypes.c_char_p, VP]
        L.rte_cnn_save_state.argtypes = [VP, ctypes.c_char_p]
        L.rte_cnn_load_state.argtypes = [VP, ctypes.c_char_p, VP]
        L.rte_guess_features.argtypes = [VP, ctypes.c_int, VP, VP, VP, VP]
        L.rte_guess_targets.argtypes = [VP, ctypes.c_int, VP, VP, VP, VP, VP]
        L.rte_cnn_guess_apply.argtypes = [VP, VP, VP, VP, VP, VP, VP]
        L.rte_guess_load.argtypes = [ctypes.POINTER(VP), ctypes.c_char_p]
        L.rte_guess_apply.argtypes = [VP, VP, VP, VP, VP]
        L.rte_guess_destroy.argtypes = [VP]
        L.rte_batch_plan.argtypes = [VP, ctypes.c_int, ctypes.POINTER(VP)]
        for name in ("rte_cnn_create", "rte_cnn_destroy", "rte_cnn_forward", "rte_cnn_train_step", "rte_cnn_layer",
                     "rte_cnn_sync_weights", "rte_cnn_save", "rte_cnn_load", "rte_cnn_save_state", "rte_cnn_load_state", "rte_guess_features",
                     "rte_guess_targets", "rte_cnn_guess_apply", "rte_guess_load", "rte_guess_apply",
                     "rte_guess_destroy", "rte_batch_plan"):
            getattr(L, name).restype = ctypes.c_int
        L.rte_status_str.argtypes = [ctypes.c_int]
        L.rte_status_str.restype = ctypes.c_char_p
        L.rte_last_error.restype = ctypes.c_char_p
        for name in ("rte_plan_create", "rte_apply_K", "rte_apply_A", "rte_apply_K32", "rte_apply_K64e",
                     "rte_apply_precond32", "rte_rhs",
                     "rte_solve",
                     "rte_solve_host", "rte_plan_info", "rte_plan_cell_weights", "rte_destroy"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _status_str(s):
    try:
        return lib().rte_status_str(int(s)).decode()
    except Exception:
        return "status %d" % s


def _check(st, where, allow=()):
    if st != RTE_OK and st not in allow:
        raise RteError(st, where, lib().rte_last_error().decode())
    return st


INNER = {"gmres": 0, "minres": 1}


MODE_MIX = {"auto": 0, "direct": 1, "fft": 2}


def make_opts(prec="fp64", tol=1e-8, restart=40, maxit=2000, inner_tol=1e-4, use_guess=0, q_policy=0,
              inner_solver="gmres", precond=0, precond_lmax=0, mode_mix=0):
    return rte_opts(PREC[prec] if isinstance(prec, str) else int(prec), tol, restart, maxit, inner_tol,
                    int(use_guess), int(q_policy),
                    INNER[inner_solver] if isinstance(inner_solver, str) else int(inner_solver), int(precond),
                    int(precond_lmax), MODE_MIX[mode_mix] if isinstance(mode_mix, str) else int(mode_mix))


def rte_plan_create(dim, n, h, mu_t, mu_s, L, sigma_hat, opts=None, stream=0):
    g = rte_grid(dim, (ctypes.c_int * 3)(n, n, n))
    sig = (ctypes.c_double * (L + 1))(*[float(v) for v in sigma_hat[:L + 1]])
    out = VP()
    st = lib().rte_plan_create(ctypes.byref(out), g, h, mu_t, mu_s, L, sig,
                               ctypes.byref(opts) if opts is not None else None, VP(stream))
    _check(st, "rte_plan_create")
    return out


def rte_apply_K(plan, x, y, stream=0):
    _check(lib().rte_apply_K(plan, VP(x), VP(y), VP(stream)), "rte_apply_K")


def rte_apply_A(plan, x, y, stream=0):
    _check(lib().rte_apply_A(plan, VP(x), VP(y), VP(stream)), "rte_apply_A")


def rte_apply_K64e(plan, x, y, stream=0):
    _check(lib().rte_apply_K64e(plan, VP(x), VP(y), VP(stream)), "rte_apply_K64e")


def rte_apply_K32(plan, x, y, stream=0):
    _check(lib().rte_apply_K32(plan, VP(x), VP(y), VP(stream)), "rte_apply_K32")


def rte_inhom_create(n, h, mu_t, stream=0):
    """mu_t: n*n cell values (x fastest), host."""
    import numpy as _np
    arr = _np.ascontiguousarray(mu_t, dtype=_np.float64).reshape(-1)
    if arr.size != n * n:
        raise ValueError("mu_t must hold n*n values")
    out = VP()
    _check(lib().rte_inhom_create(ctypes.byref(out), int(n), float(h),
                                  arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), VP(stream)),
           "rte_inhom_create")
    return out


def rte_inhom_apply32(op, x, y, stream=0):
    _check(lib().rte_inhom_apply32(op, VP(x), VP(y), VP(stream)), "rte_inhom_apply32")


def rte_inhom_apply64(op, x, y, stream=0):
    _check(lib().rte_inhom_apply64(op, VP(x), VP(y), VP(stream)), "rte_inhom_apply64")


def rte_inhom_diag(op, count):
    out = (ctypes.c_double * count)()
    _check(lib().rte_inhom_diag(op, out), "rte_inhom_diag")
    return list(out)


def rte_inhom_destroy(op):
    lib().rte_inhom_destroy(op)


def rte_aniso3d_create(n, h, mu_t, mu_s, L, sigma_hat, stream=0):
    sh = (ctypes.c_double * (L + 1))(*[float(v) for v in sigma_hat])
    out = VP()
    _check(lib().rte_aniso3d_create(ctypes.byref(out), int(n), float(h), float(mu_t), float(mu_s), int(L), sh,
                                    VP(stream)), "rte_aniso3d_create")
    return out


def rte_aniso3d_info(op):
    M, Q = ctypes.c_int(), ctypes.c_int()
    _check(lib().rte_aniso3d_info(op, ctypes.byref(M), ctypes.byref(Q)), "rte_aniso3d_info")
    return M.value, Q.value


def rte_aniso3d_pair_table(L):
    M = (L + 1) ** 2
    out = (ctypes.c_int * (M * M))()
    _check(lib().rte_aniso3d_pair_table(int(L), out), "rte_aniso3d_pair_table")
    return list(out)


def rte_aniso3d_cell_weights(op, M):
    out = (ctypes.c_double * (M * M))()
    _check(lib().rte_aniso3d_cell_weights(op, out), "rte_aniso3d_cell_weights")
    return list(out)


def rte_aniso3d_apply_K(op, x, y, stream=0):
    _check(lib().rte_aniso3d_apply_K(op, VP(x), VP(y), VP(stream)), "rte_aniso3d_apply_K")


def rte_aniso3d_apply_K64e(op, x, y, stream=0):
    _check(lib().rte_aniso3d_apply_K64e(op, VP(x), VP(y), VP(stream)), "rte_aniso3d_apply_K64e")


def rte_aniso3d_apply_K32(op, x, y, stream=0):
    _check(lib().rte_aniso3d_apply_K32(op, VP(x), VP(y), VP(stream)), "rte_aniso3d_apply_K32")


def rte_aniso3d_rhs(op, f, b, stream=0):
    _check(lib().rte_aniso3d_rhs(op, VP(f), VP(b), VP(stream)), "rte_aniso3d_rhs")


def rte_aniso3d_solve(op, f, u, tol, restart, maxit, prec="fp64", stream=0):
    stats = rte_stats()
    st = lib().rte_aniso3d_solve(op, VP(f), VP(u), float(tol), int(restart), int(maxit), PREC[prec],
                                 ctypes.byref(stats), VP(stream))
    _check(st, "rte_aniso3d_solve", allow=(RTE_ENOCONV,))
    d = stats.as_dict()
    d["status"] = st
    return d


def rte_aniso3d_destroy(op):
    lib().rte_aniso3d_destroy(op)


def rte_precond_info(plan):
    lmax = ctypes.c_int()
    _check(lib().rte_precond_info(plan, ctypes.byref(lmax)), "rte_precond_info")
    return lmax.value


def rte_apply_precond32(plan, x, y, stream=0):
    _check(lib().rte_apply_precond32(plan, VP(x), VP(y), VP(stream)), "rte_apply_precond32")


def rte_rhs(plan, f, b, stream=0):
    _check(lib().rte_rhs(plan, VP(f), VP(b), VP(stream)), "rte_rhs")


def rte_solve(plan, f, u, opts=None, stream=0):
    stats = rte_stats()
    st = lib().rte_solve(plan, VP(f), VP(u), ctypes.byref(opts) if opts is not None else None,
                         ctypes.byref(stats), VP(stream))
    _check(st, "rte_solve", allow=(RTE_ENOCONV,))
    d = stats.as_dict()
    d["status"] = st
    return d


def rte_solve_host(plan, f_host, u_host, opts=None, stream=0):
    stats = rte_stats()
    st = lib().rte_solve_host(plan, VP(f_host), VP(u_host), ctypes.byref(opts) if opts is not None else None,
                              ctypes.byref(stats), VP(stream))
    _check(st, "rte_solve_host", allow=(RTE_ENOCONV,))
    d = stats.as_dict()
    d["status"] = st
    return d


def rte_plan_info(plan):
    n, Q, L, nr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_long()
    _check(lib().rte_plan_info(plan, ctypes.byref(n), ctypes.byref(Q), ctypes.byref(L), ctypes.byref(nr)),
           "rte_plan_info")
    return dict(n=n.value, Q=Q.value, L=L.value, nreal=nr.value)


def rte_plan_cell_weights(plan, count):
    out = (ctypes.c_double * count)()
    _check(lib().rte_plan_cell_weights(plan, out), "rte_plan_cell_weights")
    return list(out)


def rte_time_passes(plan, inner, reps, stream=0, npass=3):
    out = (ctypes.c_double * npass)()
    _check(lib().rte_time_passes(plan, int(inner), int(reps), out, VP(stream)), "rte_time_passes")
    return list(out)


def rte_kernel_launches():
    return int(lib().rte_kernel_launches())


def rte_apply_K_noalloc(n, h, mu_t, mu_s, L, sigma_hat, x, y, stream=0):
    sig = (ctypes.c_double * (L + 1))(*[float(v) for v in sigma_hat[:L + 1]])
    _check(lib().rte_apply_K_noalloc(int(n), float(h), float(mu_t), float(mu_s), int(L), sig, VP(x), VP(y),
                                     VP(stream)), "rte_apply_K_noalloc")


def rte_debug_fail_alloc(k):
    """Make the k-th library allocation from now fail (0: none); returns the
    allocations since the previous call and the live (device, host) counts."""
    seen, dev, host = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
    _check(lib().rte_debug_fail_alloc(int(k), ctypes.byref(seen), ctypes.byref(dev), ctypes.byref(host)),
           "rte_debug_fail_alloc")
    return seen.value, dev.value, host.value


def rte_noalloc_scratch_bytes():
    return int(lib().rte_noalloc_scratch_bytes())


def rte_batch_create(instances, opts=None, stream=0):
    """instances: sequence of dicts with n, h, mu_t, mu_s, sigma_hat (and optional q, rows_per_block)."""
    count = len(instances)
    descs = (rte_instance_desc * count)()
    keep = []
    for i, d in enumerate(instances):
        sig = [float(v) for v in d["sigma_hat"]]
        arr = (ctypes.c_double * len(sig))(*sig)
        keep.append(arr)
        descs[i] = rte_instance_desc(int(d["n"]), float(d["h"]), float(d["mu_t"]), float(d["mu_s"]), len(sig) - 1,
                                     arr, int(d.get("q", 0)), int(d.get("rows_per_block", 0)))
    out = VP()
    st = lib().rte_batch_create(ctypes.byref(out), count, descs, ctypes.byref(opts) if opts is not None else None,
                                VP(stream))
    _check(st, "rte_batch_create")
    return out


def rte_batch_layout(batch, count):
    f = (ctypes.c_long * (count + 1))()
    u = (ctypes.c_long * (count + 1))()
    _check(lib().rte_batch_layout(batch, f, u), "rte_batch_layout")
    return list(f), list(u)


def rte_batch_solve_packed(batch, count, f_packed, u_packed, stream=0):
    stats = (rte_stats * count)()
    ms = ctypes.c_double()
    st = lib().rte_batch_solve_packed(batch, VP(f_packed), VP(u_packed), stats, ctypes.byref(ms), VP(stream))
    _check(st, "rte_batch_solve_packed", allow=(RTE_ENOCONV,))
    return st, [x.as_dict() for x in stats], ms.value


def rte_batch_solve(batch, f_ptrs, u_ptrs, stream=0):
    """f_ptrs, u_ptrs: sequences of device pointers, one per instance."""
    count = len(f_ptrs)
    fa = (VP * count)(*[VP(int(p)) for p in f_ptrs])
    ua = (VP * count)(*[VP(int(p)) for p in u_ptrs])
    stats = (rte_stats * count)()
    st = lib().rte_batch_solve(batch, fa, ua, stats, VP(stream))
    _check(st, "rte_batch_solve", allow=(RTE_ENOCONV,))
    return st, [x.as_dict() for x in stats]


def rte_batch_destroy(batch):
    _check(lib().rte_batch_destroy(batch), "rte_batch_destroy")


def rte_autotune(n, L, prec="mixed_fp32", reps=20, stream=0):
    q, rb, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().rte_autotune(int(n), int(L), PREC[prec] if isinstance(prec, str) else int(prec), int(reps),
                              ctypes.byref(q), ctypes.byref(rb), ctypes.byref(ms), VP(stream)), "rte_autotune")
    return q.value, rb.value, ms.value


def rte_batch_plan(batch, i):
    out = VP()
    _check(lib().rte_batch_plan(batch, int(i), ctypes.byref(out)), "rte_batch_plan")
    return out


def rte_cnn_create(cin=16, width=64, depth=6, cout=16, seed=0, stream=0):
    out = VP()
    _check(lib().rte_cnn_create(ctypes.byref(out), cin, width, depth, cout, seed, VP(stream)), "rte_cnn_create")
    return out


def rte_cnn_destroy(net):
    _check(lib().rte_cnn_destroy(net), "rte_cnn_destroy")


def rte_cnn_forward(net, X, B, H, W, y, stream=0):
    _check(lib().rte_cnn_forward(net, VP(X), B, H, W, VP(y), VP(stream)), "rte_cnn_forward")


def rte_cnn_train_step(net, X, T, B, H, W, used, lr, want_loss=True, stream=0):
    loss = ctypes.c_float()
    _check(lib().rte_cnn_train_step(net, VP(X), VP(T), B, H, W, used, float(lr),
                                    ctypes.byref(loss) if want_loss else None, VP(stream)), "rte_cnn_train_step")
    return loss.value


def rte_cnn_layer(net, l):
    ci, co = ctypes.c_int(), ctypes.c_int()
    w, b, gw, gb = VP(), VP(), VP(), VP()
    _check(lib().rte_cnn_layer(net, l, ctypes.byref(ci), ctypes.byref(co), ctypes.byref(w), ctypes.byref(b),
                               ctypes.byref(gw), ctypes.byref(gb)), "rte_cnn_layer")
    return dict(cin=ci.value, cout=co.value, w=w.value, b=b.value, gw=gw.value, gb=gb.value)


def rte_cnn_sync_weights(net, stream=0):
    _check(lib().rte_cnn_sync_weights(net, VP(stream)), "rte_cnn_sync_weights")


def rte_cnn_save(net, path):
    _check(lib().rte_cnn_save(net, str(path).encode()), "rte_cnn_save")


def rte_cnn_load(net, path, stream=0):
    _check(lib().rte_cnn_load(net, str(path).encode(), VP(stream)), "rte_cnn_load")


def rte_cnn_save_state(net, path):
    _check(lib().rte_cnn_save_state(net, str(path).encode()), "rte_cnn_save_state")


def rte_cnn_load_state(net, path, stream=0):
    _check(lib().rte_cnn_load_state(net, str(path).encode(), VP(stream)), "rte_cnn_load_state")


def rte_guess_features(plan, cin, f, b, X, stream=0):
    _check(lib().rte_guess_features(plan, cin, VP(f), VP(b), VP(X), VP(stream)), "rte_guess_features")


def rte_guess_targets(plan, cout, f, u, b, T, stream=0):
    _check(lib().rte_guess_targets(plan, cout, VP(f), VP(u), VP(b), VP(T), VP(stream)), "rte_guess_targets")


def rte_cnn_guess_apply(net, plan, f, b_out, Xs, u0, stream=0):
    _check(lib().rte_cnn_guess_apply(net, plan, VP(f), VP(b_out), VP(Xs), VP(u0), VP(stream)),
           "rte_cnn_guess_apply")


def rte_guess_load(path):
    out = VP()
    _check(lib().rte_guess_load(ctypes.byref(out), str(path).encode()), "rte_guess_load")
    return out


def rte_guess_apply(guess, plan, f, u0, stream=0):
    _check(lib().rte_guess_apply(guess, plan, VP(f), VP(u0), VP(stream)), "rte_guess_apply")


def rte_guess_destroy(guess):
    _check(lib().rte_guess_destroy(guess), "rte_guess_destroy")


def rte_destroy(plan):
    _check(lib().rte_destroy(plan), "rte_destroy")


def rte_status_str(s):
    return _status_str(s)


def rte_last_error():
    return lib().rte_last_error().decode()
