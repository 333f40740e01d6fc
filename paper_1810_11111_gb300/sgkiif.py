"""Thin ctypes binding of libsgkiif (C ABI in include/sgkiif.h).

The module-level ``sgk_*`` callables are the C entry points with their
argument types declared; the classes below only marshal arguments (device
buffers are passed as raw pointers, e.g. ``tensor.data_ptr()``) and turn
non-zero status codes into ``SgkError``.  Every computation runs in the CUDA
library; if the library is not built, using it raises.
"""
import ctypes
import os

import numpy as np

SGK_OK, SGK_EINVAL, SGK_ENOMEM, SGK_EUNSUPPORTED, SGK_ENEWTON, SGK_ETIMEOUT, SGK_ECUDA = range(7)
SGK_FP64, SGK_MIXED = 0, 1
SGK_PERIODIC, SGK_DIRICHLET0 = 0, 1
SGK_IIF2 = 2
SGK_IIF3 = 3
SGK_IIF_MAX_ORDER = 6
SGK_PEAK_FP32_FMA, SGK_PEAK_FP64_FMA = 0, 1
SGK_REACTION_QUADRATURE, SGK_REACTION_INTERP = 0, 1
REACTION_FORMS = {"quadrature": SGK_REACTION_QUADRATURE, "interp": SGK_REACTION_INTERP}
MAX_SPECIES = 4

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsgkiif.so")

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_i32_p = ctypes.POINTER(ctypes.c_int32)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)


class sgk_reaction(ctypes.Structure):
    _fields_ = [("nspecies", ctypes.c_int), ("nmono", ctypes.c_int), ("species", _c_int_p),
                ("coef", _c_double_p), ("exps", _c_int_p)]


class sgk_newton_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("inner_max", ctypes.c_int), ("gmres_restart", ctypes.c_int)]


class sgk_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("newton_iters", ctypes.c_int64), ("inner_iters", ctypes.c_int64),
                ("krylov_calls", ctypes.c_int64), ("krylov_breakdowns", ctypes.c_int64),
                ("last_m_eff", ctypes.c_int), ("last_newton_residual", ctypes.c_double),
                ("last_krylov_err_est", ctypes.c_double), ("max_krylov_err_est", ctypes.c_double),
                ("krylov_substeps", ctypes.c_int), ("krylov_refinements", ctypes.c_int64)]


class sgk_init(ctypes.Structure):
    _fields_ = [("coeffs", _c_double_p), ("nterms", ctypes.c_int), ("amp", _c_double_p), ("wavenum", _c_int_p),
                ("kind", _c_int_p), ("const_term", ctypes.c_double)]


class sgk_request(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_int), ("nspecies", ctypes.c_int),
                ("bc", ctypes.c_int), ("kappa", _c_double_p), ("reaction", sgk_reaction),
                ("krylov_m", ctypes.c_int), ("dt", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("precision", ctypes.c_int), ("init", sgk_init * MAX_SPECIES),
                ("krylov_tol", ctypes.c_double), ("krylov_max_substeps", ctypes.c_int),
                ("reaction_form", ctypes.c_int)]


class sgk_result_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nspecies", ctypes.c_int), ("dof", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("est_bytes", ctypes.c_int64), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("worker", ctypes.c_int),
                ("newton_iters", ctypes.c_int64), ("inner_iters", ctypes.c_int64), ("error", ctypes.c_char * 160),
                ("krylov_err_est", ctypes.c_double)]


class sgk_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("reserved_bytes", ctypes.c_int64),
                ("peak_reserved_bytes", ctypes.c_int64), ("max_concurrent", ctypes.c_int)]


_P = ctypes.c_void_p
_SIGS = {
    "sgk_ctx_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.c_int]),
    "sgk_ctx_destroy": (ctypes.c_int, [_P]),
    "sgk_last_error": (ctypes.c_char_p, [_P]),
    "sgk_ctx_launch_count": (ctypes.c_int64, [_P]),
    "sgk_binary_arch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "sgk_alu_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sgk_ctx_profile": (ctypes.c_int, [_P, ctypes.c_uint]),
    "sgk_ctx_profile_read": (ctypes.c_int, [_P, _c_double_p, _c_i64_p]),
    "sgk_index_build": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "sgk_index_destroy": (ctypes.c_int, [_P]),
    "sgk_index_dof": (ctypes.c_int64, [_P]),
    "sgk_dof": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "sgk_estimate_work": (ctypes.c_double, [ctypes.c_int] * 6),
    "sgk_partition": (ctypes.c_int, [ctypes.c_int, _c_double_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "sgk_index_ntuples": (ctypes.c_int64, [_P]),
    "sgk_index_export": (ctypes.c_int, [_P, _c_i32_p, _c_i64_p, ctypes.c_int64]),
    "sgk_index_lookup": (ctypes.c_int, [_P, _c_i32_p, ctypes.c_int64, _c_i64_p]),
    "sgk_operator_assemble": (ctypes.c_int, [_P, _P, _c_double_p, ctypes.c_int, ctypes.c_double,
                                             ctypes.POINTER(_P)]),
    "sgk_operator_assemble_full": (ctypes.c_int, [_P, _P, _c_double_p, ctypes.c_int, ctypes.c_double,
                                                  ctypes.POINTER(_P)]),
    "sgk_operator_destroy": (ctypes.c_int, [_P]),
    "sgk_operator_madds": (ctypes.c_int64, [_P]),
    "sgk_operator_export_1d": (ctypes.c_int, [_P, _c_double_p, ctypes.c_int64]),
    "sgk_matvec": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "sgk_project_separable": (ctypes.c_int, [_P, _P, ctypes.c_int, _c_double_p, _c_int_p, _c_int_p,
                                             ctypes.c_double, _P]),
    "sgk_dirichlet_load": (ctypes.c_int, [_P, _P, _c_double_p, ctypes.c_double, ctypes.c_int, _c_double_p, _c_int_p,
                                          _c_int_p, ctypes.c_double, _P]),
    "sgk_solver_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(sgk_reaction),
                                         ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.POINTER(sgk_newton_opts), ctypes.POINTER(_P)]),
    "sgk_solver_create_form": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(sgk_reaction),
                                              ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              ctypes.POINTER(sgk_newton_opts), ctypes.c_int, ctypes.POINTER(_P)]),
    "sgk_interp_factors_1d": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int64]),
    "sgk_solver_destroy": (ctypes.c_int, [_P]),
    "sgk_solver_set_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    "sgk_solver_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "sgk_solver_get_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, ctypes.c_int]),
    "sgk_solver_set_source": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "sgk_iif_alpha": (ctypes.c_int, [ctypes.c_int, _P]),
    "sgk_cross_blocks_1d": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int64]),
    "sgk_solver_step_async": (ctypes.c_int, [_P, ctypes.c_int]),
    "sgk_solver_wait": (ctypes.c_int, [_P]),
    "sgk_solver_set_time": (ctypes.c_int, [_P, ctypes.c_double]),
    "sgk_solver_get_time": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "sgk_solver_set_krylov_substeps": (ctypes.c_int, [_P, ctypes.c_int]),
    "sgk_solver_set_krylov_tolerance": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int]),
    "sgk_solver_stats": (ctypes.c_int, [_P, ctypes.POINTER(sgk_stats)]),
    "sgk_reaction_eval": (ctypes.c_int, [_P, _P, _P]),
    "sgk_jacobian_apply": (ctypes.c_int, [_P, _P, _P, _P]),
    "sgk_krylov_expv": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _c_int_p]),
    "sgk_krylov_export": (ctypes.c_int, [_P, _c_double_p, _c_double_p, ctypes.c_int64]),
    "sgk_expm_e1": (ctypes.c_int, [_P, ctypes.c_int, _c_double_p, ctypes.c_double, _c_double_p]),
    "sgk_expm_e1_noalloc": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_double, _P, _P]),
    "sgk_estimate_bytes": (ctypes.c_int64, [ctypes.c_int] * 7),
    "sgk_server_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                         ctypes.POINTER(_P)]),
    "sgk_server_set_engine": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "sgk_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(sgk_request), _c_i64_p]),
    "sgk_server_poll": (ctypes.c_int, [_P, ctypes.c_int64]),
    "sgk_server_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(sgk_result_info),
                                       _c_double_p, ctypes.c_int64]),
    "sgk_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(sgk_server_stats)]),
    "sgk_server_destroy": (ctypes.c_int, [_P]),
    "sgk_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "sgk_batch_add": (ctypes.c_int, [_P, ctypes.POINTER(sgk_request), _c_int_p]),
    "sgk_batch_step": (ctypes.c_int, [_P, ctypes.c_int, _c_int_p]),
    "sgk_batch_dof": (ctypes.c_int64, [_P, ctypes.c_int]),
    "sgk_batch_count": (ctypes.c_int, [_P]),
    "sgk_batch_get_state": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _c_double_p, ctypes.c_int64]),
    "sgk_batch_destroy": (ctypes.c_int, [_P]),
    "sgk_batch_stats": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(sgk_stats)]),
    "sgk_batch_set_fused": (ctypes.c_int, [_P, ctypes.c_int]),
    "sgk_batch_launches": (ctypes.c_int64, [_P]),
}
EXPM_NOALLOC_MAX_M = 64

_lib = None


def load():
    """Load libsgkiif.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsgkiif.so is not built (run __graft_entry__.build()); no fallback exists")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
            globals()[name] = fn
        _lib = lib
    return _lib


def exported_symbols():
    return sorted(_SIGS)


class SgkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libsgkiif status %d: %s" % (code, msg))
        self.code = code


def _dptr(arr):
    return arr.ctypes.data_as(_c_double_p)


def _iptr(arr):
    return arr.ctypes.data_as(_c_int_p)


class Context:
    def __init__(self, device=0, stream=None, precision=SGK_FP64):
        load()
        self.h = _P()
        rc = sgk_ctx_create(ctypes.byref(self.h), int(device), stream, int(precision))
        if rc:
            raise SgkError(rc, "sgk_ctx_create failed")
        self.precision = precision

    def check(self, rc):
        if rc:
            raise SgkError(rc, sgk_last_error(self.h).decode())

    @property
    def launches(self):
        return int(sgk_ctx_launch_count(self.h))

    KERNEL_CLASSES = ("matvec", "to_finest", "from_finest", "cell_quadrature", "reductions", "expm", "vector",
                      "arnoldi")

    def profile(self, mask):
        self.check(sgk_ctx_profile(self.h, int(mask)))

    def profile_read(self):
        """{class: (milliseconds, launches)} since the previous read."""
        ms = np.zeros(8)
        n = np.zeros(8, dtype=np.int64)
        self.check(sgk_ctx_profile_read(self.h, _dptr(ms), n.ctypes.data_as(_c_i64_p)))
        return {c: (float(ms[i]), int(n[i])) for i, c in enumerate(self.KERNEL_CLASSES)}

    def close(self):
        if self.h:
            sgk_ctx_destroy(self.h)
            self.h = _P()

    def expm_e1(self, X, tau):
        X = np.ascontiguousarray(X, dtype=np.float64)
        m = X.shape[0]
        y = np.zeros(m)
        self.check(sgk_expm_e1(self.h, m, _dptr(X), float(tau), _dptr(y)))
        return y


class IndexSet:
    def __init__(self, ctx, d, n, k):
        self.ctx, self.d, self.n, self.k = ctx, d, n, k
        self.h = _P()
        ctx.check(sgk_index_build(ctx.h, d, n, k, ctypes.byref(self.h)))
        self.dof = int(sgk_index_dof(self.h))
        self.ntuples = int(sgk_index_ntuples(self.h))

    def export(self):
        levels = np.zeros((self.ntuples, self.d), dtype=np.int32)
        offsets = np.zeros(self.ntuples + 1, dtype=np.int64)
        self.ctx.check(sgk_index_export(self.h, levels.ctypes.data_as(_c_i32_p),
                                        offsets.ctypes.data_as(_c_i64_p), self.ntuples))
        return levels, offsets

    def lookup(self, levels):
        levels = np.ascontiguousarray(levels, dtype=np.int32).reshape(-1, self.d)
        out = np.zeros(levels.shape[0], dtype=np.int64)
        self.ctx.check(sgk_index_lookup(self.h, levels.ctypes.data_as(_c_i32_p), levels.shape[0],
                                        out.ctypes.data_as(_c_i64_p)))
        return out

    def project_separable(self, amp, wavenum, kind, const, out_ptr):
        amp = np.ascontiguousarray(amp, dtype=np.float64)
        wavenum = np.ascontiguousarray(wavenum, dtype=np.int32).reshape(-1)
        kind = np.ascontiguousarray(kind, dtype=np.int32).reshape(-1)
        self.ctx.check(sgk_project_separable(self.ctx.h, self.h, len(amp), _dptr(amp), _iptr(wavenum),
                                             _iptr(kind), float(const), out_ptr))

    def dirichlet_load(self, kappa, amp, wavenum, kind, const, out_ptr, sigma=20.0):
        """Load vector of the boundary data const + sum_t amp_t prod_m g(2 pi w x_m)
        into the device array at out_ptr (dof doubles)."""
        kap = np.ascontiguousarray(kappa, dtype=np.float64)
        amp = np.ascontiguousarray(amp, dtype=np.float64)
        wavenum = np.ascontiguousarray(wavenum, dtype=np.int32).reshape(-1)
        kind = np.ascontiguousarray(kind, dtype=np.int32).reshape(-1)
        self.ctx.check(sgk_dirichlet_load(self.ctx.h, self.h, _dptr(kap), float(sigma), len(amp), _dptr(amp),
                                          _iptr(wavenum), _iptr(kind), float(const), out_ptr))

    def close(self):
        if self.h:
            sgk_index_destroy(self.h)
            self.h = _P()


class Operator:
    def __init__(self, ctx, idx, kappa, bc=SGK_PERIODIC, sigma=20.0):
        """kappa: the d diagonal entries of a diagonal diffusion tensor, or
        a full d x d symmetric positive definite tensor."""
        self.ctx, self.idx = ctx, idx
        kap = np.ascontiguousarray(kappa, dtype=np.float64)
        self.h = _P()
        if kap.ndim == 2:
            ctx.check(sgk_operator_assemble_full(ctx.h, idx.h, _dptr(kap.reshape(-1)), int(bc), float(sigma),
                                                 ctypes.byref(self.h)))
        else:
            ctx.check(sgk_operator_assemble(ctx.h, idx.h, _dptr(kap), int(bc), float(sigma), ctypes.byref(self.h)))
        self.H = (idx.k + 1) << idx.n

    def madds(self):
        return int(sgk_operator_madds(self.h))

    def export_1d(self):
        out = np.zeros((self.H, self.H))
        self.ctx.check(sgk_operator_export_1d(self.h, _dptr(out), out.size))
        return out

    def matvec(self, x_ptr, y_ptr, precision=SGK_FP64):
        self.ctx.check(sgk_matvec(self.h, x_ptr, y_ptr, int(precision)))

    def close(self):
        if self.h:
            sgk_operator_destroy(self.h)
            self.h = _P()


def reaction_struct(terms, nspecies):
    """terms: list per species of (coef, exponents) monomials."""
    species, coef, exps = [], [], []
    for s, mono in enumerate(terms):
        for c, e in mono:
            species.append(s)
            coef.append(float(c))
            exps.extend(int(v) for v in e)
    keep = (np.array(species or [0], dtype=np.int32), np.array(coef or [0.0]),
            np.array(exps or [0] * nspecies, dtype=np.int32))
    st = sgk_reaction(nspecies, len(species), _iptr(keep[0]), _dptr(keep[1]), _iptr(keep[2]))
    return st, keep


class Solver:
    def __init__(self, ctx, ops, reaction_terms, krylov_m, dt, opts=None, scheme=SGK_IIF2, reaction_form="quadrature"):
        self.ctx, self.ops = ctx, list(ops)
        self.nspecies = len(self.ops)
        self.dof = self.ops[0].idx.dof
        arr = (_P * self.nspecies)(*[o.h for o in self.ops])
        self._rx, self._keep = reaction_struct(reaction_terms, self.nspecies)
        o = None
        if opts:
            o = sgk_newton_opts(opts.get("tol", 0.0), opts.get("max_iter", 0), opts.get("inner_tol", 0.0),
                                opts.get("inner_max", 0), opts.get("gmres_restart", 0))
        self.h = _P()
        ctx.check(sgk_solver_create_form(ctx.h, self.nspecies, arr, ctypes.byref(self._rx), int(scheme),
                                         int(krylov_m), float(dt), ctypes.byref(o) if o else None,
                                         REACTION_FORMS[reaction_form], ctypes.byref(self.h)))

    def set_state(self, species, coeffs=None, dev_ptr=None):
        if dev_ptr is not None:
            self.ctx.check(sgk_solver_set_state(self.h, species, dev_ptr, 1))
        else:
            c = np.ascontiguousarray(coeffs, dtype=np.float64)
            assert c.size == self.dof
            self.ctx.check(sgk_solver_set_state(self.h, species, c.ctypes.data, 0))

    def set_source(self, species, lambdas, dev_ptr):
        """Source terms sum_m e^{lambdas[m] t} S_m of one species; dev_ptr: the
        len(lambdas) projected vectors S_m, back to back on the device."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        self.ctx.check(sgk_solver_set_source(self.h, species, int(lam.size), lam.ctypes.data if lam.size else None,
                                             dev_ptr if lam.size else None))

    def set_time(self, t):
        self.ctx.check(sgk_solver_set_time(self.h, float(t)))

    def set_krylov_substeps(self, substeps):
        """exp(tau A) v as `substeps` successive projections of tau/substeps
        (1: the paper's single projection)."""
        self.ctx.check(sgk_solver_set_krylov_substeps(self.h, int(substeps)))

    def set_krylov_tolerance(self, tol, max_substeps=64):
        """Accuracy guard of synchronous steps: double the sub-projections
        while the step's Krylov estimate is above tol (0: off)."""
        self.ctx.check(sgk_solver_set_krylov_tolerance(self.h, float(tol), int(max_substeps)))

    def get_time(self):
        t = ctypes.c_double()
        self.ctx.check(sgk_solver_get_time(self.h, ctypes.byref(t)))
        return t.value

    def get_state(self, species, dev_ptr=None):
        if dev_ptr is not None:
            self.ctx.check(sgk_solver_get_state(self.h, species, dev_ptr, self.dof, 1))
            return None
        out = np.zeros(self.dof)
        self.ctx.check(sgk_solver_get_state(self.h, species, out.ctypes.data, self.dof, 0))
        return out

    def step(self, nsteps=1):
        self.ctx.check(sgk_solver_step(self.h, int(nsteps)))

    def step_async(self, nsteps=1):
        self.ctx.check(sgk_solver_step_async(self.h, int(nsteps)))

    def wait(self):
        self.ctx.check(sgk_solver_wait(self.h))

    def stats(self):
        st = sgk_stats()
        self.ctx.check(sgk_solver_stats(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in sgk_stats._fields_}

    def reaction_eval(self, u_ptr, f_ptr):
        self.ctx.check(sgk_reaction_eval(self.h, u_ptr, f_ptr))

    def jacobian_apply(self, u_ptr, w_ptr, jw_ptr):
        self.ctx.check(sgk_jacobian_apply(self.h, u_ptr, w_ptr, jw_ptr))

    def krylov_expv(self, species, v_ptr, w_ptr):
        m = ctypes.c_int(0)
        self.ctx.check(sgk_krylov_expv(self.h, species, v_ptr, w_ptr, ctypes.byref(m)))
        return m.value

    def krylov_export(self, M):
        H = np.zeros((M + 1, M))
        V = np.zeros((M + 1, self.dof))
        self.ctx.check(sgk_krylov_export(self.h, _dptr(H), _dptr(V), V.size))
        return H, V

    def close(self):
        if self.h:
            sgk_solver_destroy(self.h)
            self.h = _P()


def dof_of(d, n, k):
    """Coefficients per species of the sparse grid (d, level n, degree k),
    from the library's host-side count (sgk_dof)."""
    load()
    v = sgk_dof(int(d), int(n), int(k))
    if v < 0:
        raise SgkError(SGK_EINVAL, "sgk_dof: d, n or k out of range")
    return int(v)


def interp_factors_1d(n, k, which):
    """Dense 1D factor of the interpolation form's collocation matrix (0: A,
    1: B, 2: B^-1, 3: A^-1) from the library's host tables (sgk_interp_factors_1d)."""
    load()
    H = (k + 1) << n
    out = np.zeros((H, H))
    rc = sgk_interp_factors_1d(int(n), int(k), int(which), _dptr(out), out.size)
    if rc != SGK_OK:
        raise SgkError(rc, "sgk_interp_factors_1d failed")
    return out


def binary_arch():
    """Architecture of the loaded device code (103 for sm_103a)."""
    load()
    a = ctypes.c_int(0)
    rc = sgk_binary_arch(ctypes.byref(a))
    if rc != SGK_OK:
        raise SgkError(rc, "sgk_binary_arch")
    return a.value


def alu_peak(device=0, kind="fp32"):
    """Measured FMA peak of the FP32 or FP64 pipe in flop/s (sgk_alu_peak)."""
    load()
    k = {"fp32": SGK_PEAK_FP32_FMA, "fp64": SGK_PEAK_FP64_FMA}[kind]
    out = ctypes.c_double(0.0)
    rc = sgk_alu_peak(int(device), k, ctypes.byref(out))
    if rc != SGK_OK:
        raise SgkError(rc, "sgk_alu_peak")
    return out.value


class Server:
    """Request loop over whole IIF2 solves (sgk_server_*): requests are
    workload dicts as in workloads.py; results are species-stacked FP64
    coefficients with the server's timing record."""

    def __init__(self, device=0, workers=4, mem_budget_bytes=0, aging_ms=0.0, engine=True, engine_max=0):
        load()
        self.h = _P()
        rc = sgk_server_create(int(device), int(workers), int(mem_budget_bytes), float(aging_ms),
                               ctypes.byref(self.h))
        if rc:
            raise SgkError(rc, "sgk_server_create failed")
        rc = sgk_server_set_engine(self.h, 1 if engine else 0, int(engine_max))
        if rc:
            raise SgkError(rc, "sgk_server_set_engine failed")

    @staticmethod
    def request(cfg, precision, init_coeffs=None):
        """sgk_request for a workload dict; init_coeffs (list per species of
        host arrays) overrides the separable initial data.  Returns the struct
        and the arrays it points to (keep them alive until submit returns)."""
        d, S = cfg["d"], len(cfg["kappas"])
        keep = []
        kap = np.ascontiguousarray(np.array(cfg["kappas"], dtype=np.float64).reshape(S * d))
        keep.append(kap)
        rx, rkeep = reaction_struct(cfg["reaction"], S)
        keep.append(rkeep)
        q = sgk_request()
        q.d, q.n, q.k, q.nspecies, q.bc = d, cfg["n"], cfg["k"], S, int(cfg.get("bc", SGK_PERIODIC))
        q.kappa = _dptr(kap)
        q.reaction = rx
        q.krylov_m, q.dt, q.nsteps, q.precision = int(cfg["M"]), float(cfg["dt"]), int(cfg["steps"]), int(precision)
        q.krylov_tol = float(cfg.get("krylov_tol", 0.0))
        q.krylov_max_substeps = int(cfg.get("krylov_max_substeps", 64))
        q.reaction_form = REACTION_FORMS[cfg.get("reaction_form", "quadrature")]
        if init_coeffs is None and any("noise_seed" in i for i in cfg["init"]):
            from .workloads import coefficient_noise
            init_coeffs = coefficient_noise(cfg["init"][0]["noise_seed"], dof_of(d, cfg["n"], cfg["k"]), S,
                                            [i["base"] for i in cfg["init"]])
        for s in range(S):
            init = cfg["init"][s]
            if init_coeffs is not None:
                c = np.ascontiguousarray(init_coeffs[s], dtype=np.float64)
                keep.append(c)
                q.init[s].coeffs = _dptr(c)
            else:
                amp = np.ascontiguousarray(init["amp"], dtype=np.float64)
                wn = np.ascontiguousarray(init["wavenum"], dtype=np.int32)
                kd = np.ascontiguousarray(init["kind"], dtype=np.int32)
                keep += [amp, wn, kd]
                q.init[s].nterms = len(amp)
                q.init[s].amp, q.init[s].wavenum, q.init[s].kind = _dptr(amp), _iptr(wn), _iptr(kd)
                q.init[s].const_term = float(init.get("const", 0.0))
        return q, keep

    def submit(self, cfg, precision=SGK_MIXED, init_coeffs=None):
        q, keep = self.request(cfg, precision, init_coeffs)
        t = ctypes.c_int64(0)
        rc = sgk_server_submit(self.h, ctypes.byref(q), ctypes.byref(t))
        if rc:
            raise SgkError(rc, "sgk_server_submit failed")
        return t.value

    def poll(self, ticket):
        return int(sgk_server_poll(self.h, int(ticket)))

    def wait(self, ticket, timeout_ms=-1.0, cap=None):
        """(result array or None, info dict) once the request has finished."""
        info = sgk_result_info()
        if cap is None:
            out = None
            rc = sgk_server_wait(self.h, int(ticket), float(timeout_ms), ctypes.byref(info), None, 0)
        else:
            out = np.zeros(int(cap))
            rc = sgk_server_wait(self.h, int(ticket), float(timeout_ms), ctypes.byref(info), _dptr(out), out.size)
        if rc:
            raise SgkError(rc, "sgk_server_wait failed")
        d = {f: getattr(info, f) for f, _ in sgk_result_info._fields_}
        d["error"] = d["error"].decode(errors="replace")
        if out is not None:
            out = out[:d["nspecies"] * d["dof"]]
        return out, d

    def stats(self):
        st = sgk_server_stats()
        sgk_server_get_stats(self.h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in sgk_server_stats._fields_}

    def close(self):
        if self.h:
            sgk_server_destroy(self.h)
            self.h = _P()


class Batch:
    """Independent IIF2 problems stepped together (sgk_batch_*); instances
    are workload dicts as for Server."""

    def __init__(self, device=0, streams=8, slice_len=0, fused=True):
        load()
        self.h = _P()
        rc = sgk_batch_create(int(device), int(streams), int(slice_len), ctypes.byref(self.h))
        if rc:
            raise SgkError(rc, "sgk_batch_create failed")
        sgk_batch_set_fused(self.h, 1 if fused else 0)
        self.nspecies = []

    def launches(self):
        """Kernels of the batched Arnoldi path so far."""
        return int(sgk_batch_launches(self.h))

    def stats(self, i):
        st = sgk_stats()
        rc = sgk_batch_stats(self.h, int(i), ctypes.byref(st))
        if rc:
            raise SgkError(rc, "sgk_batch_stats failed")
        return {f: getattr(st, f) for f, _ in sgk_stats._fields_}

    def add(self, cfg, precision=SGK_MIXED, init_coeffs=None):
        q, keep = Server.request(cfg, precision, init_coeffs)
        i = ctypes.c_int(-1)
        rc = sgk_batch_add(self.h, ctypes.byref(q), ctypes.byref(i))
        if rc:
            raise SgkError(rc, "sgk_batch_add failed")
        self.nspecies.append(len(cfg["kappas"]))
        return i.value

    def step(self, nsteps=1):
        st = (ctypes.c_int * max(1, len(self.nspecies)))()
        rc = sgk_batch_step(self.h, int(nsteps), st)
        return rc, [st[i] for i in range(len(self.nspecies))]

    def dof(self, i):
        return int(sgk_batch_dof(self.h, int(i)))

    def state(self, i):
        n = self.dof(i)
        out = []
        for s in range(self.nspecies[i]):
            a = np.zeros(n)
            rc = sgk_batch_get_state(self.h, int(i), s, _dptr(a), n)
            if rc:
                raise SgkError(rc, "sgk_batch_get_state failed")
            out.append(a)
        return out

    def close(self):
        if self.h:
            sgk_batch_destroy(self.h)
            self.h = _P()
