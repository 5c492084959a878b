"""Python binding of libusbs (include/usbs.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all arithmetic
runs in the CUDA library.  Importing this module loads ``libusbs.so`` and raises if it
has not been built (``python -m paper_2312_11801_gb300.build``): there is no fallback.
Device buffers may be passed as torch CUDA tensors (their ``data_ptr()`` is used).
"""
import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libusbs.so")

USBS_OK, USBS_EINVAL, USBS_ENOMEM, USBS_ECUDA = 0, -1, -2, -3
USBS_ETIMEOUT, USBS_ENOTCONV, USBS_EBUSY, USBS_ENUMERIC = -4, -5, -6, -7
KINDS = ["spmm", "reorth", "restart", "constraint", "small_fp64", "reduce", "sketch", "setup",
         "reorth_update", "reorth_final", "ritz"]
PRECISION_FP64, PRECISION_MIXED = 0, 1
_ERR = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENOTCONV",
        -6: "EBUSY", -7: "ENUMERIC"}


class usbs_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("rho", ctypes.c_double), ("beta", ctypes.c_double),
                ("k_c", ctypes.c_int), ("k_p", ctypes.c_int), ("r", ctypes.c_int),
                ("precision", ctypes.c_int), ("lanczos_basis", ctypes.c_int),
                ("lanczos_restarts", ctypes.c_int), ("lanczos_tol", ctypes.c_double),
                ("ipm_mu_tol", ctypes.c_double), ("ipm_max_iter", ctypes.c_int),
                ("max_alt", ctypes.c_int), ("alt_tol", ctypes.c_double),
                ("trace_hint", ctypes.c_double), ("max_iters", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("certify_restarts", ctypes.c_int), ("certify_tol", ctypes.c_double),
                ("obj_gap_tol", ctypes.c_double), ("model_value_ipm", ctypes.c_int)]


class usbs_eig_info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("matvecs", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_residual", ctypes.c_double), ("jacobi_sweeps", ctypes.c_int),
                ("reruns", ctypes.c_int)]


class usbs_step_info(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("descent", ctypes.c_int), ("n_alt", ctypes.c_int),
                ("ipm_iters", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("f_y", ctypes.c_double), ("f_cand", ctypes.c_double), ("f_hat", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("cx", ctypes.c_double), ("trx", ctypes.c_double),
                ("eta", ctypes.c_double), ("relgap", ctypes.c_double), ("relinf", ctypes.c_double),
                ("relinf_max", ctypes.c_double), ("objective", ctypes.c_double),
                ("dual_bound", ctypes.c_double), ("f_hat_closed", ctypes.c_double),
                ("ipm_iters_b1", ctypes.c_int)]


class usbs_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("descent_steps", ctypes.c_int), ("matvecs", ctypes.c_longlong),
                ("last", usbs_step_info), ("certifications", ctypes.c_int),
                ("cert_residual", ctypes.c_double), ("obj_gap", ctypes.c_double)]


class usbs_server_params(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int),
                ("cache_entries", ctypes.c_int), ("dry_run", ctypes.c_int),
                ("solver", usbs_params)]


class usbs_completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("parent_id", ctypes.c_int64),
                ("status", ctypes.c_int), ("warm", ctypes.c_int), ("iters", ctypes.c_int),
                ("slot", ctypes.c_int), ("objective", ctypes.c_double),
                ("dual_bound", ctypes.c_double), ("relgap", ctypes.c_double),
                ("relinf", ctypes.c_double), ("t_arrival", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_finish", ctypes.c_double),
                ("bytes", ctypes.c_uint64)]


class usbs_server_stats_t(ctypes.Structure):
    _fields_ = [("used_bytes", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64), ("pending", ctypes.c_int),
                ("running", ctypes.c_int), ("peak_running", ctypes.c_int), ("cached", ctypes.c_int),
                ("finished", ctypes.c_int64), ("rejected", ctypes.c_int64)]


def _struct_dict(s):
    out = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        out[name] = _struct_dict(v) if isinstance(v, ctypes.Structure) else v
    return out


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("usbs_params_default", None, [ctypes.POINTER(usbs_params)]),
    ("usbs_abi_version", ctypes.c_int, []),
    ("usbs_last_error", ctypes.c_char_p, [_P]),
    ("usbs_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, _I64, _I32, _D,
                                   ctypes.c_int64, ctypes.c_int64, _I32, _I32, _I32, _D, _D, _U8,
                                   _F, ctypes.POINTER(usbs_params)]),
    ("usbs_destroy", ctypes.c_int, [_P]),
    ("usbs_extreme_eigs", ctypes.c_int, [_P, _D, ctypes.c_int, _D, _D,
                                         ctypes.POINTER(usbs_eig_info)]),
    ("usbs_step", ctypes.c_int, [_P, ctypes.POINTER(usbs_step_info)]),
    ("usbs_solve", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(usbs_result)]),
    ("usbs_get_sketch", ctypes.c_int, [_P, _F, _F, _D]),
    ("usbs_nystrom_round", ctypes.c_int, [_P, _D, _D, _D, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int8)]),
    ("usbs_qap_round", ctypes.c_int, [_P, ctypes.c_int, _D, _D, _D, _D, _I32, ctypes.POINTER(ctypes.c_int)]),
    ("usbs_get_dual", ctypes.c_int, [_P, _D]),
    ("usbs_get_primal_constraints", ctypes.c_int, [_P, _D]),
    ("usbs_state_size", ctypes.c_int64, [_P]),
    ("usbs_get_state", ctypes.c_int, [_P, _D]),
    ("usbs_set_state", ctypes.c_int, [_P, _D]),
    ("usbs_grow", ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.c_int64, _I64, _I32, _D,
                                 ctypes.c_int64, ctypes.c_int64, _I32, _I32, _I32, _D, _D, _U8, _F]),
    ("usbs_op_matmul", ctypes.c_int, [_P, _P, _P, _P]),
    ("usbs_op_constraint_eval", ctypes.c_int, [_P, _P, _P, _P]),
    ("usbs_op_sketch_update", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_double]),
    ("usbs_sketch_update_static", ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _P, _P, _P, _P,
                                                 ctypes.c_double, _P]),
    ("usbs_profile", ctypes.c_int, [_P, ctypes.c_int]),
    ("usbs_kernel_stats", ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_longlong), _D]),
    ("usbs_launch_count", ctypes.c_longlong, [_P]),
    ("usbs_selftest_tile_wait", ctypes.c_int, [ctypes.c_int]),
    ("usbs_selftest_tf32_round", ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("usbs_instance_bytes", ctypes.c_uint64, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
    ("usbs_server_params_default", None, [ctypes.POINTER(usbs_server_params)]),
    ("usbs_server_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(usbs_server_params)]),
    ("usbs_server_submit", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _I64, _I32,
                                          _D, ctypes.c_int64, ctypes.c_int64, _I32, _I32, _I32, _D, _D,
                                          _U8, _F, ctypes.c_double, ctypes.c_double]),
    ("usbs_server_poll", ctypes.c_int, [_P, ctypes.POINTER(usbs_completion), ctypes.c_int, ctypes.c_int]),
    ("usbs_server_get_stats", ctypes.c_int, [_P, ctypes.POINTER(usbs_server_stats_t)]),
    ("usbs_server_destroy", ctypes.c_int, [_P]),
    ("usbs_batch_solve", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(usbs_result), ctypes.POINTER(ctypes.c_int)]),
    ("usbs_scaling", ctypes.c_int, [_P, _D, _D]),
    ("usbs_dims", ctypes.c_int, [_P, _I64, _I64, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)]),
]

_lib = None


def load(path=LIB_PATH):
    """Open libusbs.so (raises OSError / RuntimeError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libusbs.so not built ({path}); run python -m paper_2312_11801_gb300.build")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class USBSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"usbs error {code} ({_ERR.get(code, '?')}): {msg}")
        self.code = code


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dev(t):
    """Device address of a torch tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _check(rc, ctx_ptr=None, allow=()):
    if rc != USBS_OK and rc not in allow:
        msg = load().usbs_last_error(ctx_ptr)
        raise USBSError(rc, msg.decode() if msg else "")
    return rc


def params_default(**overrides):
    p = usbs_params()
    load().usbs_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream            # torch.cuda.Stream
        setattr(p, k, v)
    return p


class Context:
    """Owns one usbs_ctx (usbs_create / usbs_destroy)."""

    def __init__(self, ptr, n, m, r):
        self.ptr = ptr
        self.n, self.m, self.r = n, m, r

    @property
    def handle(self):
        return self.ptr

    def close(self):
        if self.ptr:
            load().usbs_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _problem_arrays(prob):
    return (np.ascontiguousarray(prob.C_rowptr, np.int64), np.ascontiguousarray(prob.C_col, np.int32),
            np.ascontiguousarray(prob.C_val, np.float64), np.ascontiguousarray(prob.A_con, np.int32),
            np.ascontiguousarray(prob.A_i, np.int32), np.ascontiguousarray(prob.A_j, np.int32),
            np.ascontiguousarray(prob.A_val, np.float64), np.ascontiguousarray(prob.b, np.float64),
            np.ascontiguousarray(prob.is_ineq, np.uint8))


def usbs_create(prob, psi=None, params=None, **overrides):
    """usbs_create from an ``instances.Problem``; returns a Context."""
    lib = load()
    p = params if params is not None else params_default(**overrides)
    if params is not None:
        for k, v in overrides.items():
            setattr(p, k, v)
    rp, cc, cv, ac, ai, aj, av, b, iq = _problem_arrays(prob)
    psi_a = None if psi is None else np.ascontiguousarray(psi, np.float32)
    out = ctypes.c_void_p()
    rc = lib.usbs_create(ctypes.byref(out), prob.n, _ptr(rp, ctypes.c_int64), _ptr(cc, ctypes.c_int32),
                         _ptr(cv, ctypes.c_double), prob.m, len(ac), _ptr(ac, ctypes.c_int32),
                         _ptr(ai, ctypes.c_int32), _ptr(aj, ctypes.c_int32), _ptr(av, ctypes.c_double),
                         _ptr(b, ctypes.c_double), _ptr(iq, ctypes.c_uint8),
                         None if psi_a is None else _ptr(psi_a, ctypes.c_float), ctypes.byref(p))
    _check(rc, None)
    return Context(out, prob.n, prob.m, p.r)


def usbs_destroy(ctx):
    ctx.close()


def usbs_extreme_eigs(ctx, y=None, kc=None, want_vecs=True):
    """Top eigenpairs of (C - A*(y)) / ||C||_F; y in problem units (None = current)."""
    lib = load()
    kcap = ctypes.c_int()
    lib.usbs_dims(ctx.ptr, None, None, ctypes.byref(kcap), None, None, None)
    kc = kcap.value if kc is None else kc
    evals = np.zeros(kc)
    evecs = np.zeros((ctx.n, kc)) if want_vecs else None
    ya = None if y is None else np.ascontiguousarray(y, np.float64)
    info = usbs_eig_info()
    _check(lib.usbs_extreme_eigs(ctx.ptr, None if ya is None else _ptr(ya, ctypes.c_double), kc,
                                 _ptr(evals, ctypes.c_double),
                                 None if evecs is None else _ptr(evecs, ctypes.c_double),
                                 ctypes.byref(info)), ctx.ptr)
    return evals, evecs, _struct_dict(info)


def usbs_step(ctx):
    info = usbs_step_info()
    _check(load().usbs_step(ctx.ptr, ctypes.byref(info)), ctx.ptr)
    return _struct_dict(info)


def usbs_solve(ctx, warm_start=False, tol=1e-3):
    res = usbs_result()
    _check(load().usbs_solve(ctx.ptr, int(bool(warm_start)), float(tol), ctypes.byref(res)), ctx.ptr,
           allow=(USBS_ENOTCONV,))
    return _struct_dict(res)


def usbs_get_sketch(ctx):
    P = np.zeros((ctx.n, ctx.r), np.float32)
    Psi = np.zeros((ctx.n, ctx.r), np.float32)
    sc = np.zeros(2)
    _check(load().usbs_get_sketch(ctx.ptr, _ptr(P, ctypes.c_float), _ptr(Psi, ctypes.c_float),
                                  _ptr(sc, ctypes.c_double)), ctx.ptr)
    return P, Psi, sc


def usbs_nystrom_round(ctx, want_u=True, want_signs=True):
    """Rank-r reconstruction X_hat = U diag(lam) U^T of the primal from the sketch and the
    best sign-vector cut over the columns of U (problem units).  Returns
    (lam, U or None, values, best, signs or None)."""
    lam = np.zeros(ctx.r)
    vals = np.zeros(ctx.r)
    U = np.zeros((ctx.n, ctx.r)) if want_u else None
    z = np.zeros(ctx.n, np.int8) if want_signs else None
    best = ctypes.c_int(-1)
    _check(load().usbs_nystrom_round(ctx.ptr, _ptr(lam, ctypes.c_double),
                                     None if U is None else _ptr(U, ctypes.c_double),
                                     _ptr(vals, ctypes.c_double), ctypes.byref(best),
                                     None if z is None else _ptr(z, ctypes.c_int8)), ctx.ptr)
    return lam, U, vals, best.value, z


def usbs_qap_round(ctx, W, D):
    """QAP rounding of the sketch: (costs, scores, perms (r x nq), best column)."""
    W = np.ascontiguousarray(W, np.float64)
    D = np.ascontiguousarray(D, np.float64)
    nq = W.shape[0]
    costs = np.zeros(ctx.r)
    scores = np.zeros(ctx.r)
    perms = np.zeros((ctx.r, nq), np.int32)
    best = ctypes.c_int()
    _check(load().usbs_qap_round(ctx.ptr, nq, _ptr(W, ctypes.c_double), _ptr(D, ctypes.c_double),
                                 _ptr(costs, ctypes.c_double), _ptr(scores, ctypes.c_double),
                                 _ptr(perms, ctypes.c_int32), ctypes.byref(best)), ctx.ptr)
    return costs, scores, perms, best.value


def usbs_get_dual(ctx):
    y = np.zeros(ctx.m)
    _check(load().usbs_get_dual(ctx.ptr, _ptr(y, ctypes.c_double)), ctx.ptr)
    return y


def usbs_get_primal_constraints(ctx):
    ax = np.zeros(ctx.m)
    _check(load().usbs_get_primal_constraints(ctx.ptr, _ptr(ax, ctypes.c_double)), ctx.ptr)
    return ax


def usbs_get_state(ctx):
    st = np.zeros(load().usbs_state_size(ctx.ptr))
    _check(load().usbs_get_state(ctx.ptr, _ptr(st, ctypes.c_double)), ctx.ptr)
    return st


def usbs_set_state(ctx, state):
    st = np.ascontiguousarray(state, np.float64)
    _check(load().usbs_set_state(ctx.ptr, _ptr(st, ctypes.c_double)), ctx.ptr)


def usbs_grow(ctx, prob, psi=None):
    lib = load()
    rp, cc, cv, ac, ai, aj, av, b, iq = _problem_arrays(prob)
    psi_a = None if psi is None else np.ascontiguousarray(psi, np.float32)
    out = ctypes.c_void_p()
    rc = lib.usbs_grow(ctx.ptr, ctypes.byref(out), prob.n, _ptr(rp, ctypes.c_int64),
                       _ptr(cc, ctypes.c_int32), _ptr(cv, ctypes.c_double), prob.m, len(ac),
                       _ptr(ac, ctypes.c_int32), _ptr(ai, ctypes.c_int32), _ptr(aj, ctypes.c_int32),
                       _ptr(av, ctypes.c_double), _ptr(b, ctypes.c_double), _ptr(iq, ctypes.c_uint8),
                       None if psi_a is None else _ptr(psi_a, ctypes.c_float))
    _check(rc, ctx.ptr)
    return Context(out, prob.n, prob.m, ctx.r)


def usbs_scaling(ctx):
    c, t = ctypes.c_double(), ctypes.c_double()
    _check(load().usbs_scaling(ctx.ptr, ctypes.byref(c), ctypes.byref(t)), ctx.ptr)
    return c.value, t.value


def usbs_dims(ctx):
    n, m = ctypes.c_int64(), ctypes.c_int64()
    k, r, prec, J = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().usbs_dims(ctx.ptr, ctypes.byref(n), ctypes.byref(m), ctypes.byref(k),
                            ctypes.byref(r), ctypes.byref(prec), ctypes.byref(J)), ctx.ptr)
    return {"n": n.value, "m": m.value, "k_c": k.value, "r": r.value, "precision": prec.value,
            "basis": J.value}


def usbs_op_matmul(ctx, y_scaled_dev, X_dev, Y_dev):
    _check(load().usbs_op_matmul(ctx.ptr, _dev(y_scaled_dev), _dev(X_dev), _dev(Y_dev)), ctx.ptr)


def usbs_op_constraint_eval(ctx, V_dev, S_dev, z_dev):
    _check(load().usbs_op_constraint_eval(ctx.ptr, _dev(V_dev), _dev(S_dev), _dev(z_dev)), ctx.ptr)


def usbs_op_sketch_update(ctx, V_dev, S_dev, Psi_dev, P_dev, eta):
    _check(load().usbs_op_sketch_update(ctx.ptr, _dev(V_dev), _dev(S_dev), _dev(Psi_dev),
                                        _dev(P_dev), float(eta)), ctx.ptr)


def usbs_profile(ctx, on=True):
    _check(load().usbs_profile(ctx.ptr, int(bool(on))), ctx.ptr)


def usbs_kernel_stats(ctx):
    """{kind name: (total device ms, launches, algorithmic bytes)} since profiling on."""
    out = {}
    for k, name in enumerate(KINDS):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        by = ctypes.c_double()
        _check(load().usbs_kernel_stats(ctx.ptr, k, ctypes.byref(ms), ctypes.byref(n),
                                        ctypes.byref(by)), ctx.ptr)
        out[name] = (ms.value, n.value, by.value)
    return out


def usbs_launch_count(ctx):
    return int(load().usbs_launch_count(ctx.ptr))


def usbs_selftest_tile_wait(deliver):
    """The staged tiles' bounded wait run alone; returns the status code (no exception)."""
    return load().usbs_selftest_tile_wait(int(bool(deliver)))


def usbs_selftest_tf32_round(x):
    """The FP32 tiles' TF32 rounding of x and cvt.rna.tf32.f32's, as uint32 bit arrays."""
    x = np.ascontiguousarray(x, np.float32)
    ours = np.zeros(x.size, np.uint32)
    ref = np.zeros(x.size, np.uint32)
    _check(load().usbs_selftest_tf32_round(x.size, _ptr(x, ctypes.c_float), _ptr(ours, ctypes.c_uint32),
                                           _ptr(ref, ctypes.c_uint32)), None)
    return ours, ref


def usbs_sketch_update_static(n, r, V_dev, S_dev, Psi_dev, P_dev, eta, stream=None):
    """Context-free sketch update that allocates nothing (see include/usbs.h)."""
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().usbs_sketch_update_static(int(n), int(r), _dev(V_dev), _dev(S_dev),
                                            _dev(Psi_dev), _dev(P_dev), float(eta), st), None)


def usbs_instance_bytes(n, nnzC, m, nnzA, r=0, precision=PRECISION_MIXED):
    return int(load().usbs_instance_bytes(n, nnzC, m, nnzA, r, precision))


def usbs_server_params_default(**overrides):
    p = usbs_server_params()
    load().usbs_server_params_default(ctypes.byref(p))
    solver = overrides.pop("solver", None)
    for k, v in overrides.items():
        setattr(p, k, v)
    for k, v in (solver or {}).items():
        setattr(p.solver, k, v)
    return p


class Server:
    """Owns one usbs_server (usbs_server_create / usbs_server_destroy)."""

    def __init__(self, ptr, r):
        self.ptr = ptr
        self.r = r

    def close(self):
        if self.ptr:
            load().usbs_server_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def usbs_server_create(**params):
    p = usbs_server_params_default(**params)
    out = ctypes.c_void_p()
    _check(load().usbs_server_create(ctypes.byref(out), ctypes.byref(p)), None)
    return Server(out, p.solver.r)


def usbs_server_submit(srv, request_id, prob, parent_id=-1, psi=None, tol=1e-3, fake_service_s=0.0):
    rp, cc, cv, ac, ai, aj, av, b, iq = _problem_arrays(prob)
    psi_a = None if psi is None else np.ascontiguousarray(psi, np.float32)
    _check(load().usbs_server_submit(
        srv.ptr, int(request_id), int(parent_id), prob.n, _ptr(rp, ctypes.c_int64),
        _ptr(cc, ctypes.c_int32), _ptr(cv, ctypes.c_double), prob.m, len(ac), _ptr(ac, ctypes.c_int32),
        _ptr(ai, ctypes.c_int32), _ptr(aj, ctypes.c_int32), _ptr(av, ctypes.c_double),
        _ptr(b, ctypes.c_double), _ptr(iq, ctypes.c_uint8),
        None if psi_a is None else _ptr(psi_a, ctypes.c_float), float(tol), float(fake_service_s)), None)


def usbs_server_poll(srv, max_items=64, wait_ms=0):
    buf = (usbs_completion * max_items)()
    k = load().usbs_server_poll(srv.ptr, buf, max_items, int(wait_ms))
    _check(min(k, 0), None)
    return [_struct_dict(buf[i]) for i in range(k)]


def usbs_server_get_stats(srv):
    st = usbs_server_stats_t()
    _check(load().usbs_server_get_stats(srv.ptr, ctypes.byref(st)), None)
    return _struct_dict(st)


def usbs_server_destroy(srv):
    srv.close()


def usbs_batch_solve(ctxs, tol=1e-3, max_concurrency=8):
    n = len(ctxs)
    arr = (ctypes.c_void_p * n)(*[c.ptr.value if isinstance(c.ptr, ctypes.c_void_p) else c.ptr for c in ctxs])
    res = (usbs_result * n)()
    st = (ctypes.c_int * n)()
    rc = load().usbs_batch_solve(arr, n, float(tol), int(max_concurrency), res, st)
    _check(rc, None, allow=(USBS_ENOTCONV,))
    return [_struct_dict(res[i]) for i in range(n)], list(st)
