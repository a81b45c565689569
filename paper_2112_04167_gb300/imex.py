"""Thin ctypes binding of the C ABI in include/imex.h (argument marshalling only).

Every function here forwards to the CUDA library ``_lib/libimexgb.so``; there is
no CPU implementation behind it.  Arrays may be NumPy arrays (host memory, FP64,
C-contiguous) or CUDA tensors exposing ``data_ptr()`` (device memory, FP64,
contiguous).  Errors raise ``ImexError`` with the library's message.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libimexgb.so")

OK, EINVAL, ENOMEM, ENOTCONV, EUNSTABLE, ECUDA = range(6)
FP64, MIXED, MIXED_FAST = 0, 1, 2
POISSON_SIPG, POISSON_CONSISTENT = 0, 1
FLOW_NONE, FLOW_TG2D, FLOW_TG3D, FLOW_TGTRAVEL, FLOW_VV = 0, 1, 2, 3, 4
NU_CONST, NU_VARXYT, NU_VELOCITY, NU_FIELD = 0, 1, 2, 3
FORCE_NONE, FORCE_TGTRAVEL_VARNU, FORCE_VV = 0, 1, 2
SPACE_VELOCITY, SPACE_PRESSURE = 0, 1
ARITH_FP64, ARITH_FP32, ARITH_FF = 0, 1, 3
PRECOND_JACOBI, PRECOND_PMG = 0, 1
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTCONV", 4: "EUNSTABLE", 5: "ECUDA"}


class ImexError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class imex_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("P", C.c_int), ("nelem", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("periodic", C.c_int * 3), ("precision", C.c_int),
                ("poisson", C.c_int), ("tol", C.c_double), ("maxit", C.c_int), ("inner_tol", C.c_double),
                ("vmax", C.c_double), ("stream", C.c_void_p)]


class imex_server_desc(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("precision", C.c_int), ("poisson", C.c_int), ("tol", C.c_double),
                ("maxit", C.c_int), ("vmax", C.c_double), ("keep_results", C.c_int)]


class imex_request(C.Structure):
    _fields_ = [("dim", C.c_int), ("P", C.c_int), ("nelem", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("periodic", C.c_int * 3), ("flow", C.c_int),
                ("flow_params", C.c_double * 8), ("nu_kind", C.c_int), ("nu_params", C.c_double * 8),
                ("bc_kind", C.c_int), ("bc_params", C.c_double * 8), ("f_kind", C.c_int),
                ("f_params", C.c_double * 8), ("t0", C.c_double), ("dt", C.c_double), ("nsteps", C.c_int)]


class imex_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("active", C.c_longlong), ("queued", C.c_longlong), ("ticks", C.c_longlong),
                ("p50_tick_ms", C.c_double), ("p99_tick_ms", C.c_double), ("mean_tick_ms", C.c_double),
                ("dof_stages", C.c_double), ("busy_s", C.c_double), ("footprint_bytes", C.c_double),
                ("max_footprint_bytes", C.c_double), ("budget_bytes", C.c_double), ("groups", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class imex_stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("stages", C.c_longlong), ("poisson_solves", C.c_int),
                ("helmholtz_solves", C.c_int), ("poisson_iters", C.c_longlong),
                ("helmholtz_iters", C.c_longlong), ("refinements", C.c_int), ("max_poisson_res", C.c_double),
                ("max_helmholtz_res", C.c_double), ("div_norm", C.c_double), ("max_velocity", C.c_double),
                ("last_call_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "imex_create": [C.POINTER(imex_mesh_desc), C.POINTER(_P)],
    "imex_destroy": [_P],
    "imex_last_error": [_P],
    "imex_sizes": [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)],
    "imex_set_tableau": [_P, C.c_int, _P, _P, _P, _P, _P],
    "imex_set_tableau_named": [_P, C.c_char_p],
    "imex_set_sdc": [_P, C.c_int, C.c_int, C.c_char_p],
    "imex_set_bdf2": [_P],
    "imex_set_stabilization": [_P, C.c_double, C.c_double],
    "imex_stabilize": [_P, _P, C.c_double, _P, C.c_int],
    "imex_set_viscosity_const": [_P, C.c_double],
    "imex_set_viscosity_model": [_P, C.c_int, _P, C.c_int],
    "imex_set_viscosity_field": [_P, _P, C.c_int],
    "imex_set_boundary": [_P, C.c_int, _P, C.c_int],
    "imex_set_forcing": [_P, C.c_int, _P, C.c_int],
    "imex_set_state": [_P, C.c_double, _P, C.c_int],
    "imex_init_flow": [_P, C.c_int, _P, C.c_int, C.c_double],
    "imex_step": [_P, C.c_double, C.c_int],
    "imex_get_velocity": [_P, _P, C.c_int],
    "imex_get_pressure": [_P, _P, C.c_int],
    "imex_get_time": [_P, _D],
    "imex_get_stats": [_P, C.POINTER(imex_stats)],
    "imex_op_sipg": [_P, C.c_int, _P, _P, C.c_int, C.c_double, C.c_double, _P, _P, C.c_int, C.c_int, C.c_int],
    "imex_op_sipg_diag": [_P, C.c_int, _P, C.c_double, C.c_double, _P, C.c_int],
    "imex_op_div": [_P, _P, _P, C.c_int, _P, C.c_int, C.c_int],
    "imex_op_grad": [_P, _P, _P, C.c_int, C.c_int],
    "imex_op_conv": [_P, _P, _P, _P, C.c_int, C.c_int],
    "imex_op_graddiv": [_P, _P, _P, _P, _P, C.c_int, C.c_int],
    "imex_solve_poisson": [_P, _P, _P, C.c_int],
    "imex_set_pressure_precond": [_P, C.c_int, _P, C.c_int],
    "imex_pmg_info": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), _D],
    "imex_op_pmg_vcycle": [_P, _P, _P, _P, C.c_int, C.c_int],
    "imex_solve_helmholtz": [_P, _P, _P, C.c_double, _P, _P, C.c_int],
    "imex_eval_field": [_P, C.c_int, C.c_int, _P, C.c_int, C.c_double, _P, _P, C.c_int],
    "imex_reduce": [_P, C.c_int, _P, _P, C.c_longlong, _D, C.c_int],
    "imex_dissipation": [_P, _D],
    "imex_energy_spectrum": [_P, C.c_int, C.c_int, _D],
    "imex_reduce_noalloc": [C.c_int, _P, _P, C.c_longlong, _D, _P],
    "imex_profile": [_P, C.c_int],
    "imex_profile_read": [_P, C.c_int, C.POINTER(C.c_longlong), _D],
    "imex_profile_work": [_P, C.c_int, _D, _D, C.POINTER(C.c_int)],
    "imex_launch_count": [],
    "imex_set_apply_variant": [C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_int],
    "imex_tuning_info": [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                         C.POINTER(C.c_longlong), C.POINTER(C.c_int), _D],
    "imex_batch_create": [C.POINTER(_P), C.c_int, C.POINTER(_P)],
    "imex_batch_destroy": [_P],
    "imex_batch_last_error": [_P],
    "imex_batch_groups": [_P],
    "imex_batch_step": [_P, _D, C.c_int],
    "imex_batch_get_velocity": [_P, C.c_int, _P, C.c_int],
    "imex_batch_get_pressure": [_P, C.c_int, _P, C.c_int],
    "imex_batch_get_time": [_P, C.c_int, _D],
    "imex_batch_get_stats": [_P, C.POINTER(imex_stats)],
    "imex_batch_group_info": [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                              C.POINTER(imex_stats), _D],
    "imex_server_create": [C.POINTER(imex_server_desc), C.POINTER(_P)],
    "imex_server_destroy": [_P],
    "imex_server_last_error": [_P],
    "imex_server_submit": [_P, C.POINTER(imex_request), C.POINTER(C.c_longlong)],
    "imex_server_tick": [_P, C.POINTER(C.c_int)],
    "imex_server_poll": [_P, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_int), _D],
    "imex_server_result": [_P, C.c_longlong, _D],
    "imex_server_get_stats": [_P, C.POINTER(imex_server_stats)],
    "imex_request_footprint": [C.POINTER(imex_request), _D],
}
REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED = range(4)
(PROF_PRESSURE_F32, PROF_PRESSURE_F64, PROF_HELMHOLTZ_F32, PROF_HELMHOLTZ_F64, PROF_CONV, PROF_PCG_PERSIST,
 PROF_PMG_APPLY, PROF_PMG_VEC, PROF_CG_STEP, PROF_CG_DIR, PROF_DIV, PROF_GRAD, PROF_DERIV,
 PROF_PMG_APPLY_COARSE) = range(14)
PROF_NAMES = ["sipg_pressure_f32", "sipg_pressure_f64", "sipg_helmholtz_f32", "sipg_helmholtz_f64", "conv",
              "pcg_persist_f32", "pmg_apply", "pmg_vec", "cg_step", "cg_dir", "div", "grad", "deriv",
              "pmg_apply_coarse"]
REDUCE_DOT, REDUCE_SUM, REDUCE_MAXABS = range(3)


def exported_symbols():
    return sorted(_SIGS)


def tuning_info():
    """Launch shapes chosen by the apply tuner: one dict per tuned (d, N, precision, elements)."""
    lib = load()
    out = []
    n = lib.imex_tuning_info(-1, None, None, None, None, None, None)
    for i in range(n):
        d, N, f32, v = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ne = C.c_longlong()
        us = (C.c_double * 4)()
        lib.imex_tuning_info(i, C.byref(d), C.byref(N), C.byref(f32), C.byref(ne), C.byref(v), us)
        out.append({"d": d.value, "N": N.value, "fp32": bool(f32.value), "elements": ne.value, "variant": v.value,
                    "us": [round(x, 2) for x in us]})
    return out


def set_apply_variant(d, N, fp32, elements, variant):
    """Fix the launch shape of the periodic constant-viscosity apply (imex_set_apply_variant)."""
    st = load().imex_set_apply_variant(d, N, int(bool(fp32)), elements, variant)
    if st != OK:
        raise ImexError(st, "imex_set_apply_variant failed")


def launch_count():
    """Kernels launched by the library so far (all contexts)."""
    return int(load().imex_launch_count())


NOALLOC_MAX_N = 256 * 65536


def reduce_noalloc(op, x, y=None, stream=None):
    """imex_reduce_noalloc: the same reduction as Context.reduce without a context or any
    device allocation.  x, y: contiguous float64 CUDA tensors; stream: CUDA stream handle."""
    n = int(x.numel())
    px, dev, _a = _arr(x, n)
    if not dev:
        raise ValueError("reduce_noalloc takes device tensors")
    py, _, _b = _arr(y, n) if y is not None else (None, 0, None)
    out = C.c_double()
    st = load().imex_reduce_noalloc(op, px, py, n, C.byref(out), stream)
    if st != OK:
        raise ImexError(st, "imex_reduce_noalloc failed")
    return out.value


def load(path=None):
    """Load the CUDA library; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CUDA library {p} is missing: build it with paper_2112_04167_gb300.build.build()")
    lib = C.CDLL(p)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = {"imex_last_error": C.c_char_p, "imex_destroy": None, "imex_batch_last_error": C.c_char_p,
                     "imex_batch_destroy": None, "imex_server_last_error": C.c_char_p,
                     "imex_server_destroy": None, "imex_launch_count": C.c_longlong}.get(name, C.c_int)
    _lib = lib
    return lib


def _arr(a, n=None, writable=False):
    """(pointer, on_device, keepalive) for a NumPy array or a CUDA tensor."""
    if a is None:
        return None, 0, None
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        if not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise ValueError("device tensors must be contiguous float64")
        if n is not None and a.numel() < n:
            raise ValueError(f"tensor has {a.numel()} elements, need {n}")
        return C.c_void_p(a.data_ptr()), 1, a
    arr = np.asarray(a)
    if arr.dtype != np.float64 or not arr.flags.c_contiguous or (writable and not arr.flags.writeable):
        if writable:
            raise ValueError("output arrays must be writable C-contiguous float64")
        arr = np.ascontiguousarray(arr, dtype=np.float64)
    if n is not None and arr.size < n:
        raise ValueError(f"array has {arr.size} elements, need {n}")
    return arr.ctypes.data_as(C.c_void_p), 0, arr


def _params(p):
    if p is None or len(p) == 0:
        return None, 0, None
    arr = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    return arr.ctypes.data_as(C.c_void_p), len(arr), arr


class Context:
    """One flow instance on the GPU (wraps imex_ctx*)."""

    def __init__(self, dim, P, nelem, lo, hi, periodic, precision=FP64, poisson=POISSON_SIPG, tol=1e-12,
                 maxit=5000, inner_tol=0.0, vmax=0.0, stream=None):
        lib = load()
        d = imex_mesh_desc()
        d.dim, d.P = dim, P
        for k in range(3):
            d.nelem[k] = int(nelem[k]) if k < len(nelem) else 1
            d.lo[k] = float(lo[k]) if k < len(lo) else 0.0
            d.hi[k] = float(hi[k]) if k < len(hi) else 1.0
            d.periodic[k] = int(bool(periodic[k])) if k < len(periodic) else 1
        d.precision, d.poisson, d.tol, d.maxit, d.inner_tol, d.vmax = precision, poisson, tol, maxit, inner_tol, vmax
        d.stream = stream
        h = _P()
        st = lib.imex_create(C.byref(d), C.byref(h))
        if st != OK:
            raise ImexError(st, "imex_create failed")
        self._h = h
        self.dim = dim
        self.P = P
        nv, npr = C.c_longlong(), C.c_longlong()
        lib.imex_sizes(h, C.byref(nv), C.byref(npr))
        self.nvel, self.npres = nv.value, npr.value

    def _check(self, st):
        if st != OK:
            raise ImexError(st, load().imex_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().imex_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- configuration -------------------------------------------------------
    def set_tableau_named(self, name):
        self._check(load().imex_set_tableau_named(self._h, name.encode()))

    def set_tableau(self, c, AI, bI, AE, bE):
        s = len(c)
        arrs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in (c, AI, bI, AE, bE)]
        ptrs = [a.ctypes.data_as(C.c_void_p) for a in arrs]
        self._check(load().imex_set_tableau(self._h, s, *ptrs))

    def set_sdc(self, M, K, predictor="EULER"):
        self._check(load().imex_set_sdc(self._h, M, K, predictor.encode()))

    def set_stabilization(self, zeta_d, zeta_c):
        self._check(load().imex_set_stabilization(self._h, zeta_d, zeta_c))

    def stabilize(self, v, dt):
        out = np.empty((self.dim, self.nvel))
        pv, dev, _a = _arr(v, self.dim * self.nvel)
        po, _, _b = _arr(out, self.dim * self.nvel, writable=True)
        self._check(load().imex_stabilize(self._h, pv, dt, po, dev))
        return out

    def set_bdf2(self):
        self._check(load().imex_set_bdf2(self._h))

    def set_viscosity_const(self, nu):
        self._check(load().imex_set_viscosity_const(self._h, nu))

    def set_viscosity_model(self, kind, params):
        p, n, _k = _params(params)
        self._check(load().imex_set_viscosity_model(self._h, kind, p, n))

    def set_viscosity_field(self, nu):
        p, dev, _k = _arr(nu, self.nvel)
        self._check(load().imex_set_viscosity_field(self._h, p, dev))

    def set_boundary(self, kind, params=()):
        p, n, _k = _params(params)
        self._check(load().imex_set_boundary(self._h, kind, p, n))

    def set_forcing(self, kind, params=()):
        p, n, _k = _params(params)
        self._check(load().imex_set_forcing(self._h, kind, p, n))

    def set_state(self, t, v):
        p, dev, _k = _arr(v, self.dim * self.nvel)
        self._check(load().imex_set_state(self._h, t, p, dev))

    def init_flow(self, kind, params=(), t=0.0):
        p, n, _k = _params(params)
        self._check(load().imex_init_flow(self._h, kind, p, n, t))

    # --- stepping and queries ----------------------------------------------
    def step(self, dt, nsteps=1):
        self._check(load().imex_step(self._h, dt, nsteps))

    def get_velocity(self, out=None):
        if out is None:
            out = np.empty((self.dim, self.nvel))
        p, dev, _k = _arr(out, self.dim * self.nvel, writable=True)
        self._check(load().imex_get_velocity(self._h, p, dev))
        return out

    def get_pressure(self, out=None):
        if out is None:
            out = np.empty(self.npres)
        p, dev, _k = _arr(out, self.npres, writable=True)
        self._check(load().imex_get_pressure(self._h, p, dev))
        return out

    def time(self):
        t = C.c_double()
        self._check(load().imex_get_time(self._h, C.byref(t)))
        return t.value

    def stats(self):
        s = imex_stats()
        self._check(load().imex_get_stats(self._h, C.byref(s)))
        return s.as_dict()

    # --- operators -------------------------------------------------------------
    def op_sipg(self, x, space=SPACE_VELOCITY, nsys=1, alpha=0.0, beta=1.0, nu=None, g=None, minv=0,
                precision=ARITH_FP64):
        """precision: ARITH_FP64, ARITH_FP32 (== MIXED) or ARITH_FF."""
        n = (self.nvel if space == SPACE_VELOCITY else self.npres) * nsys
        out = np.empty(n)
        px, dev, _a = _arr(x, n)
        pn, _, _b = _arr(nu, self.nvel)
        pg, _, _c = _arr(g, n)
        py, _, _d = _arr(out, n, writable=True)
        self._check(load().imex_op_sipg(self._h, space, px, py, nsys, alpha, beta, pn, pg, minv, precision, dev))
        return out

    def op_sipg_diag(self, space=SPACE_VELOCITY, alpha=0.0, beta=1.0, nu=None):
        n = self.nvel if space == SPACE_VELOCITY else self.npres
        out = np.empty(n)
        pn, dev, _b = _arr(nu, self.nvel)
        py, _, _d = _arr(out, n, writable=True)
        self._check(load().imex_op_sipg_diag(self._h, space, py, alpha, beta, pn, 0))
        return out

    def op_div(self, v, w=None, mode=0, arith=ARITH_FP64):
        out = np.empty(self.npres)
        pv, _, _a = _arr(v, self.dim * self.nvel)
        pw, _, _b = _arr(w, self.dim * self.nvel)
        pb, _, _c = _arr(out, self.npres, writable=True)
        self._check(load().imex_op_div(self._h, pv, pw, mode, pb, arith, 0))
        return out

    def op_grad(self, psi, arith=ARITH_FP64):
        out = np.empty((self.dim, self.nvel))
        pp, _, _a = _arr(psi, self.npres)
        po, _, _b = _arr(out, self.dim * self.nvel, writable=True)
        self._check(load().imex_op_grad(self._h, pp, po, arith, 0))
        return out

    def op_conv(self, v, vb=None, arith=ARITH_FP64):
        out = np.empty((self.dim, self.nvel))
        pv, _, _a = _arr(v, self.dim * self.nvel)
        pb, _, _b = _arr(vb, self.dim * self.nvel)
        po, _, _c = _arr(out, self.dim * self.nvel, writable=True)
        self._check(load().imex_op_conv(self._h, pv, pb, po, arith, 0))
        return out

    def op_graddiv(self, v, nu=None, with_fd2=False, arith=ARITH_FP64):
        fd3 = np.empty((self.dim, self.nvel))
        fd2 = np.empty((self.dim, self.nvel)) if with_fd2 else None
        pv, _, _a = _arr(v, self.dim * self.nvel)
        pn, _, _b = _arr(nu, self.nvel)
        p3, _, _c = _arr(fd3, self.dim * self.nvel, writable=True)
        p2, _, _d = _arr(fd2, self.dim * self.nvel, writable=True) if with_fd2 else (None, 0, None)
        self._check(load().imex_op_graddiv(self._h, pv, pn, p3, p2, arith, 0))
        return (fd3, fd2) if with_fd2 else fd3

    def set_pressure_precond(self, kind, params=()):
        p, n, _k = _params(params)
        self._check(load().imex_set_pressure_precond(self._h, kind, p, n))

    def pmg_info(self):
        """(N per level, Chebyshev upper bounds per level) of the pressure V-cycle."""
        nl = C.c_int()
        N = (C.c_int * 4)()
        lm = (C.c_double * 4)()
        self._check(load().imex_pmg_info(self._h, C.byref(nl), N, lm))
        return list(N[:nl.value]), list(lm[:nl.value])

    def op_pmg_vcycle(self, r, lmax=None, arith=ARITH_FP64):
        out = np.empty(self.npres)
        pr, dev, _a = _arr(r, self.npres)
        pl, _, _b = _params(lmax)
        po, _, _c = _arr(out, self.npres, writable=True)
        self._check(load().imex_op_pmg_vcycle(self._h, pr, po, pl, arith, dev))
        return out

    def solve_poisson(self, b):
        out = np.empty(self.npres)
        pb, _, _a = _arr(b, self.npres)
        po, _, _b = _arr(out, self.npres, writable=True)
        self._check(load().imex_solve_poisson(self._h, pb, po, 0))
        return out

    def solve_helmholtz(self, g, gamma, nu=None, vb=None):
        out = np.empty((self.dim, self.nvel))
        pg, _, _a = _arr(g, self.dim * self.nvel)
        pn, _, _b = _arr(nu, self.nvel)
        pv, _, _c = _arr(vb, self.dim * self.nvel)
        po, _, _d = _arr(out, self.dim * self.nvel, writable=True)
        self._check(load().imex_solve_helmholtz(self._h, pg, pn, gamma, pv, po, 0))
        return out

    def reduce(self, op, x, y=None):
        """Device reduction of x (and y) -- DOT, SUM or MAXABS -- with FP64 accumulation."""
        n = int(x.numel()) if hasattr(x, "numel") else int(np.asarray(x).size)
        px, dev, _a = _arr(x, n)
        py, _, _b = _arr(y, n) if y is not None else (None, 0, None)
        out = C.c_double()
        self._check(load().imex_reduce(self._h, op, px, py, n, C.byref(out), dev))
        return out.value

    def dissipation(self):
        """Viscous dissipation rate of the current velocity (Sec. 4.3)."""
        e = C.c_double()
        self._check(load().imex_dissipation(self._h, C.byref(e)))
        return e.value

    def energy_spectrum(self, M, kmax):
        """E(0..kmax-1) of the current velocity on an M^d regular grid (Sec. 4.3)."""
        out = np.empty(kmax)
        self._check(load().imex_energy_spectrum(self._h, M, kmax, out.ctypes.data_as(_D)))
        return out

    def profile(self, enable=True):
        self._check(load().imex_profile(self._h, int(enable)))

    def profile_read(self, cls):
        n, ms = C.c_longlong(), C.c_double()
        self._check(load().imex_profile_read(self._h, cls, C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def profile_work(self, cls):
        """(algorithmic bytes, flops, arith of the last launch) of a profiled kernel class."""
        b, f, a = C.c_double(), C.c_double(), C.c_int()
        self._check(load().imex_profile_work(self._h, cls, C.byref(b), C.byref(f), C.byref(a)))
        return b.value, f.value, a.value

    def eval_field(self, what, kind, params=(), t=0.0, v=None):
        ncomp = 1 if what == 1 else self.dim
        out = np.empty((ncomp, self.nvel))
        pp, n, _k = _params(params)
        pv, _, _a = _arr(v, self.dim * self.nvel)
        po, _, _b = _arr(out, ncomp * self.nvel, writable=True)
        self._check(load().imex_eval_field(self._h, what, kind, pp, n, t, pv, po, 0))
        return out


class Batch:
    """Instances advanced together (wraps imex_batch*): imex_batch_create groups the
    contexts into union meshes; each step advances every instance by its own dt."""

    def __init__(self, contexts):
        lib = load()
        n = len(contexts)
        hs = (_P * n)(*[c._h for c in contexts])
        self.sizes = [(c.dim, c.nvel, c.npres) for c in contexts]
        h = _P()
        st = lib.imex_batch_create(hs, n, C.byref(h))
        if st != OK:
            raise ImexError(st, "imex_batch_create failed")
        self._h = h
        self.n = n

    def _check(self, st):
        if st != OK:
            raise ImexError(st, load().imex_batch_last_error(self._h).decode())

    @property
    def groups(self):
        return int(load().imex_batch_groups(self._h))

    def step(self, dt, nsteps=1):
        arr = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.n,)))
        self._check(load().imex_batch_step(self._h, arr.ctypes.data_as(_D), nsteps))

    def get_velocity(self, i, out=None):
        if not 0 <= i < self.n:
            raise IndexError(f"instance {i} of {self.n}")
        d, nv, _ = self.sizes[i]
        if out is None:
            out = np.empty(d * nv)
        p, dev, _k = _arr(out, d * nv, writable=True)
        self._check(load().imex_batch_get_velocity(self._h, i, p, dev))
        return out

    def get_pressure(self, i, out=None):
        if not 0 <= i < self.n:
            raise IndexError(f"instance {i} of {self.n}")
        _, _, npr = self.sizes[i]
        if out is None:
            out = np.empty(npr)
        p, dev, _k = _arr(out, npr, writable=True)
        self._check(load().imex_batch_get_pressure(self._h, i, p, dev))
        return out

    def time(self, i):
        t = C.c_double()
        self._check(load().imex_batch_get_time(self._h, i, C.byref(t)))
        return t.value

    def stats(self):
        s = imex_stats()
        self._check(load().imex_batch_get_stats(self._h, C.byref(s)))
        return s.as_dict()

    def group_info(self, q):
        n, P, nv, ms = C.c_int(), C.c_int(), C.c_longlong(), C.c_double()
        st = imex_stats()
        self._check(load().imex_batch_group_info(self._h, q, C.byref(n), C.byref(P), C.byref(nv), C.byref(st),
                                                 C.byref(ms)))
        return {"instances": n.value, "P": P.value, "nvel": nv.value, "last_ms": ms.value,
                "poisson_iters": st.poisson_iters, "poisson_solves": st.poisson_solves,
                "helmholtz_iters": st.helmholtz_iters}

    def close(self):
        if getattr(self, "_h", None):
            load().imex_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fill8(arr, vals):
    for i, v in enumerate(list(vals or ())[:8]):
        arr[i] = float(v)


class Server:
    """Continuous-batching server (wraps imex_server*): requests are admitted under an HBM
    budget and every tick advances all active requests by one step."""

    def __init__(self, budget_bytes=0.0, precision=MIXED, poisson=POISSON_SIPG, tol=1e-10, maxit=20000, vmax=0.0,
                 keep_results=False):
        d = imex_server_desc(float(budget_bytes), precision, poisson, tol, maxit, vmax, int(bool(keep_results)))
        h = _P()
        st = load().imex_server_create(C.byref(d), C.byref(h))
        if st != OK:
            raise ImexError(st, "imex_server_create failed")
        self._h = h
        self._sizes = {}

    def _check(self, st):
        if st != OK:
            raise ImexError(st, load().imex_server_last_error(self._h).decode())

    @staticmethod
    def request(dim, P, nelem, lo, hi, periodic, flow, flow_params=(), nu_kind=NU_CONST, nu_params=(),
                bc_kind=FLOW_NONE, bc_params=(), f_kind=FORCE_NONE, f_params=(), t0=0.0, dt=0.01, nsteps=1):
        """The imex_request structure of a flow request."""
        r = imex_request()
        r.dim, r.P = dim, P
        for k in range(3):
            r.nelem[k] = int(nelem[k]) if k < len(nelem) else 1
            r.lo[k] = float(lo[k]) if k < len(lo) else 0.0
            r.hi[k] = float(hi[k]) if k < len(hi) else 1.0
            r.periodic[k] = int(bool(periodic[k])) if k < len(periodic) else 1
        r.flow, r.nu_kind, r.bc_kind, r.f_kind = flow, nu_kind, bc_kind, f_kind
        _fill8(r.flow_params, flow_params)
        _fill8(r.nu_params, nu_params)
        _fill8(r.bc_params, bc_params)
        _fill8(r.f_params, f_params)
        r.t0, r.dt, r.nsteps = t0, dt, nsteps
        return r

    @staticmethod
    def footprint(**req):
        """Device bytes the request occupies once admitted (imex_request_footprint)."""
        b = C.c_double()
        st = load().imex_request_footprint(C.byref(Server.request(**req)), C.byref(b))
        if st != OK:
            raise ImexError(st, "imex_request_footprint failed")
        return b.value

    def submit(self, **req):
        r = self.request(**req)
        dim, P, nelem = req["dim"], req["P"], req["nelem"]
        i = C.c_longlong()
        self._check(load().imex_server_submit(self._h, C.byref(r), C.byref(i)))
        ne = 1
        for k in range(dim):
            ne *= int(nelem[k])
        self._sizes[i.value] = dim * ne * (P + 1) ** dim
        return i.value

    def last_error(self):
        """The server's last error message (a failed group step names its group)."""
        return load().imex_server_last_error(self._h).decode()

    def tick(self):
        a = C.c_int()
        self._check(load().imex_server_tick(self._h, C.byref(a)))
        return a.value

    def poll(self, i):
        st, n, t = C.c_int(), C.c_int(), C.c_double()
        self._check(load().imex_server_poll(self._h, i, C.byref(st), C.byref(n), C.byref(t)))
        return st.value, n.value, t.value

    def result(self, i):
        out = np.empty(self._sizes[i])
        self._check(load().imex_server_result(self._h, i, out.ctypes.data_as(_D)))
        return out

    def stats(self):
        s = imex_server_stats()
        self._check(load().imex_server_get_stats(self._h, C.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            load().imex_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
