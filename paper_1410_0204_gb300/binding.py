"""Thin ctypes binding of libmetos3d.so (include/metos3d.h): argument marshalling only.

Every step of the TMM year map runs in the library's CUDA kernels; this module converts
numpy arrays and torch CUDA tensors into the pointers and sizes of the C ABI, passes the
current torch stream, and turns status codes into exceptions.  There is no CPU path: if
the library is missing the import of a context fails.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

M3D_OK = 0
M3D_NOT_CONVERGED = 1
M3D_ERR_ARG = -1
M3D_ERR_CUDA = -2
M3D_ERR_NONFINITE = -3
M3D_ERR_TIMEOUT = -4
M3D_ERR_UNSUPPORTED = -5

OPT_YEAR_PLAN = 1
OPT_WAIT_TIMEOUT_NS = 2
OPT_TEST_WITHHOLD_TILE = 3
OPT_NTILES = 4
OPT_IMPLICIT_FORM = 5
OPT_ADJOINT_PLAN = 6
OPT_STEP_OPERATORS = 7
OPT_STEP_OPERATOR_BYTES = 8
OPT_KERNEL_TIMING = 9
OPT_LAST_KERNEL_NS = 10
OPT_TANGENT_FORM = 11
TANGENT_DUAL = 0
TANGENT_LINEARISED = 1
IMPLICIT_DENSE = 0
IMPLICIT_TRIDIAGONAL = 1
PLAN_PERSISTENT = 0
PLAN_GRAPH = 1
PLAN_RESIDENT = 2

MODEL_NONE = 0
MODEL_N = 1
MODEL_NDOP = 2
MODEL_PHY = 3
MODEL_NPZD = 5
MODEL_NTRACER = {MODEL_N: 1, MODEL_NDOP: 2, MODEL_PHY: 3, MODEL_NPZD: 5}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "metos3d.h")


class Metos3dError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("metos3d status %d: %s" % (status, msg))
        self.status = status


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int), ("ncol", C.c_int), ("col_start", C.POINTER(C.c_int)),
                ("h", C.POINTER(C.c_double)), ("zc", C.POINTER(C.c_double)),
                ("vol", C.POINTER(C.c_double)), ("lat", C.POINTER(C.c_double))]


class _Matrices(C.Structure):
    _fields_ = [("nmonth", C.c_int), ("nnz", C.c_int), ("exp_rowptr", C.POINTER(C.c_int)),
                ("exp_colidx", C.POINTER(C.c_int)), ("exp_val", C.POINTER(C.c_double)),
                ("s_imp", C.c_longlong), ("imp_blk", C.POINTER(C.c_double))]


class NewtonOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_newton", C.c_int), ("restart", C.c_int), ("max_krylov", C.c_int),
                ("jv", C.c_int), ("fd_eps", C.c_double), ("line_search", C.c_int)]


NEWTON_MAX_HIST = 64
NEWTON_MAX_TRIALS = 512


class NewtonReport(C.Structure):
    _fields_ = [("converged", C.c_int), ("newton_steps", C.c_int), ("krylov_total", C.c_int),
                ("year_maps", C.c_int), ("tangent_maps", C.c_int), ("residual0", C.c_double),
                ("residual", C.c_double), ("residuals", C.c_double * NEWTON_MAX_HIST),
                ("krylov", C.c_int * NEWTON_MAX_HIST), ("lambdas", C.c_double * NEWTON_MAX_HIST),
                ("etas", C.c_double * NEWTON_MAX_HIST), ("slopes", C.c_double * NEWTON_MAX_HIST),
                ("trials", C.c_int * NEWTON_MAX_HIST), ("ntrial", C.c_int),
                ("trial_lambdas", C.c_double * NEWTON_MAX_TRIALS), ("seconds", C.c_double),
                ("line_search_failed", C.c_int)]

    def to_dict(self):
        k = self.newton_steps
        kk = min(k, NEWTON_MAX_HIST)
        flat = list(self.trial_lambdas[:self.ntrial])
        per_step, at = [], 0
        for cnt in self.trials[:kk]:
            per_step.append(flat[at:at + cnt])
            at += cnt
        return {"converged": bool(self.converged), "newton_steps": k, "krylov_total": self.krylov_total,
                "year_maps": self.year_maps, "tangent_maps": self.tangent_maps, "residual0": self.residual0,
                "residual": self.residual, "residuals": list(self.residuals[:k + 1]),
                "krylov": list(self.krylov[:kk]), "lambdas": list(self.lambdas[:kk]),
                "etas": list(self.etas[:kk]), "slopes": list(self.slopes[:kk]), "trials": per_step,
                "seconds": self.seconds, "line_search_failed": bool(self.line_search_failed)}


JV_FD = 0
JV_TANGENT = 1


class GradientOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("max_krylov", C.c_int), ("ckpt_every", C.c_int)]


class GradientReport(C.Structure):
    _fields_ = [("converged", C.c_int), ("krylov", C.c_int), ("reverse_sweeps", C.c_int),
                ("forward_years", C.c_double), ("residual", C.c_double), ("seconds", C.c_double)]

    def to_dict(self):
        return {"converged": bool(self.converged), "krylov": self.krylov, "reverse_sweeps": self.reverse_sweeps,
                "forward_years": self.forward_years, "residual": self.residual, "seconds": self.seconds}


class _Member(C.Structure):
    _fields_ = [("model_id", C.c_int), ("nparam", C.c_int), ("u", C.POINTER(C.c_double))]


class _Model(C.Structure):
    _fields_ = [("model_id", C.c_int), ("ntracer", C.c_int), ("nparam", C.c_int),
                ("nsub", C.c_int), ("nstep", C.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmetos3d.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("libmetos3d.so is not built: run __graft_entry__.build() "
                               "or python -m paper_1410_0204_gb300.build")
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    L.metos3d_init.argtypes = [C.POINTER(vp), C.POINTER(_Grid), C.POINTER(_Matrices), C.POINTER(_Model), vp]
    L.metos3d_set_stream.argtypes = [vp, vp]
    L.metos3d_step.argtypes = [vp, C.c_int, vp, vp, vp]
    L.metos3d_year_map.argtypes = [vp, vp, vp, vp]
    L.metos3d_year_map_host.argtypes = [vp, dp, dp, dp]
    L.metos3d_mass.argtypes = [vp, vp, dp]
    L.metos3d_residual.argtypes = [vp, vp, vp, dp]
    L.metos3d_check_finite.argtypes = [vp, vp]
    L.metos3d_bgc.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                              C.c_double, C.c_double, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp,
                              C.c_int, dp, C.c_int]
    L.metos3d_info.argtypes = [vp, ip, ip, ip, ip]
    L.metos3d_last_launch_count.argtypes = [vp]
    L.metos3d_last_launch_count.restype = C.c_longlong
    L.metos3d_last_error.argtypes = [vp]
    L.metos3d_last_error.restype = C.c_char_p
    L.metos3d_free.argtypes = [vp]
    L.metos3d_free.restype = None
    L.metos3d_sync.argtypes = [vp]
    L.metos3d_set_option.argtypes = [vp, C.c_int, C.c_longlong]
    L.metos3d_get_option.argtypes = [vp, C.c_int]
    L.metos3d_get_option.restype = C.c_longlong
    L.metos3d_newton_default_options.argtypes = [C.POINTER(NewtonOptions)]
    L.metos3d_newton_default_options.restype = None
    L.metos3d_newton_solve.argtypes = [vp, vp, vp, C.POINTER(NewtonOptions), C.POINTER(NewtonReport)]
    L.metos3d_gradient_default_options.argtypes = [C.POINTER(GradientOptions)]
    L.metos3d_gradient_default_options.restype = None
    L.metos3d_periodic_gradient.argtypes = [vp, vp, vp, vp, vp, dp, C.POINTER(GradientOptions),
                                            C.POINTER(GradientReport)]
    L.metos3d_spinup.argtypes = [vp, vp, vp, C.c_int, C.c_double, dp, C.POINTER(C.c_int)]
    L.metos3d_year_tangent.argtypes = [vp, vp, vp, vp, vp, vp]
    L.metos3d_year_adjoint.argtypes = [vp, vp, vp, vp, vp, dp, C.c_int]
    L.metos3d_residual_static.argtypes = [vp, vp, C.c_longlong, vp, vp]
    L.metos3d_residual_static_error.argtypes = []
    L.metos3d_residual_static_error.restype = C.c_char_p
    L.metos3d_ensemble_init.argtypes = [C.POINTER(vp), C.POINTER(_Grid), C.POINTER(_Matrices), C.c_int,
                                        C.POINTER(_Member), C.c_int, C.c_int, vp]
    L.metos3d_ensemble_init_tangent.argtypes = [C.POINTER(vp), C.POINTER(_Grid), C.POINTER(_Matrices), C.c_int,
                                                C.POINTER(_Member), C.c_int, C.c_int, vp]
    L.metos3d_ensemble_year_adjoint.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_double), C.c_int]
    L.metos3d_ensemble_newton_solve.argtypes = [vp, vp, vp, C.POINTER(C.c_double), C.POINTER(NewtonOptions),
                                                C.POINTER(NewtonReport)]
    L.metos3d_ensemble_layout.argtypes = [vp, ip, ip, ip, ip, ip]
    L.metos3d_ensemble_set_stream.argtypes = [vp, vp]
    L.metos3d_ensemble_set_params.argtypes = [vp, C.c_int, dp]
    L.metos3d_ensemble_steps.argtypes = [vp, C.c_int, C.c_int, vp, vp]
    L.metos3d_ensemble_year_map.argtypes = [vp, vp, vp]
    L.metos3d_ensemble_set_tiling.argtypes = [vp, C.c_int, C.c_int]
    L.metos3d_ensemble_get_tiling.argtypes = [vp, ip, ip]
    L.metos3d_ensemble_autotune.argtypes = [vp, vp, C.c_int, ip, ip, dp]
    L.metos3d_ensemble_last_launch_count.argtypes = [vp]
    L.metos3d_ensemble_last_launch_count.restype = C.c_longlong
    L.metos3d_ensemble_last_error.argtypes = [vp]
    L.metos3d_ensemble_last_error.restype = C.c_char_p
    L.metos3d_ensemble_free.argtypes = [vp]
    L.metos3d_ensemble_free.restype = None
    for name in declared_symbols():
        fn = getattr(L, name)
        if name not in ("metos3d_last_error", "metos3d_free", "metos3d_last_launch_count",
                        "metos3d_residual_static_error", "metos3d_get_option",
                        "metos3d_newton_default_options", "metos3d_gradient_default_options",
                        "metos3d_ensemble_last_launch_count",
                        "metos3d_ensemble_last_error", "metos3d_ensemble_free"):
            fn.restype = C.c_int
    _lib = L
    return L


def declared_symbols():
    """Names of the functions include/metos3d.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(metos3d_[a-z_0-9]+)\s*\(", text)))


def _check(status, ctx=None):
    if status != M3D_OK:
        msg = load().metos3d_last_error(ctx).decode(errors="replace")
        raise Metos3dError(status, msg)
    return status


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _torch():
    import torch
    return torch


def _dev_ptr(t, numel, name, writable=False):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != numel:
        raise ValueError("%s must be a contiguous float64 tensor of %d elements" % (name, numel))
    return C.c_void_p(t.data_ptr())


def bgc(y, h, d, u, t=0.0, dt=1.0 / 2880, lat=0.0, insol=0.0, dayfrac=0.5, ice=0.0, wind=0.0,
        model=MODEL_NDOP, nsub=1):
    """The model interface of Section 5.2 on one column, on the GPU (host arrays)."""
    L = load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    ntr, nl = y.shape
    h = np.ascontiguousarray(h, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(y)
    _check(L.metos3d_bgc(model, t, dt, lat, insol, dayfrac, ice, wind, ntr, nl, _dp(h), _dp(d),
                         None, None, _dp(y), _dp(out), u.shape[0], _dp(u), nsub))
    return out


class Context:
    """A metos3d context on the current CUDA device (host inputs are copied at init)."""

    def __init__(self, *, col_start, h, zc, vol, lat, exp_rowptr, exp_colidx, exp_val, imp_blk,
                 model=MODEL_NDOP, ntracer=2, nparam=7, nsub=1, nstep=2880, stream=None):
        torch = _torch()
        L = load()
        self._L = L
        cs = np.ascontiguousarray(col_start, dtype=np.int32)
        self.n = int(cs[-1])
        self.ncol = int(cs.shape[0] - 1)
        self.ntracer = int(ntracer)
        self.nparam = int(nparam)
        self.nstep = int(nstep)
        h, zc, vol, lat = (np.ascontiguousarray(a, dtype=np.float64) for a in (h, zc, vol, lat))
        rp = np.ascontiguousarray(exp_rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(exp_colidx, dtype=np.int32)
        ev = np.ascontiguousarray(exp_val, dtype=np.float64)
        ib = np.ascontiguousarray(imp_blk, dtype=np.float64)
        nmonth = ev.shape[0]
        g = _Grid(self.n, self.ncol, _ip(cs), _dp(h), _dp(zc), _dp(vol), _dp(lat))
        m = _Matrices(nmonth, ci.shape[0], _ip(rp), _ip(ci), _dp(ev), ib.shape[1], _dp(ib))
        md = _Model(model, self.ntracer, self.nparam, nsub, self.nstep)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        ctx = C.c_void_p()
        _check(L.metos3d_init(C.byref(ctx), C.byref(g), C.byref(m), C.byref(md), C.c_void_p(stream.cuda_stream)))
        self._ctx = ctx

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(col_start=prob.col_start, h=prob.h, zc=prob.zc, vol=prob.vol, lat=prob.lat,
                   exp_rowptr=prob.exp_rowptr, exp_colidx=prob.exp_colidx, exp_val=prob.exp_val,
                   imp_blk=prob.imp_blk, nstep=prob.nstep, **kw)

    # ---- helpers
    def _sync_stream(self):
        torch = _torch()
        s = torch.cuda.current_stream()
        if s.cuda_stream != self._stream.cuda_stream:
            self._stream = s
            _check(self._L.metos3d_set_stream(self._ctx, C.c_void_p(s.cuda_stream)), self._ctx)

    @property
    def numel(self):
        return self.ntracer * self.n

    def new_state(self):
        torch = _torch()
        return torch.empty((self.ntracer, self.n), dtype=torch.float64, device="cuda")

    # ---- the C ABI
    def step(self, j, y_in, y_out, u):
        self._sync_stream()
        _check(self._L.metos3d_step(self._ctx, int(j), _dev_ptr(y_in, self.numel, "y_in"),
                                    _dev_ptr(y_out, self.numel, "y_out", True),
                                    _dev_ptr(u, self.nparam, "u") if self.nparam else None), self._ctx)
        return y_out

    def year_map(self, y0, y1, u):
        self._sync_stream()
        _check(self._L.metos3d_year_map(self._ctx, _dev_ptr(y0, self.numel, "y0"),
                                        _dev_ptr(y1, self.numel, "y1", True),
                                        _dev_ptr(u, self.nparam, "u") if self.nparam else None), self._ctx)
        return y1

    def year_tangent(self, y0, v, u, phi_out, jv_out):
        """phi(y0) into phi_out and phi'(y0) v into jv_out (CUDA tensors)."""
        self._sync_stream()
        _check(self._L.metos3d_year_tangent(self._ctx, _dev_ptr(y0, self.numel, "y0"), _dev_ptr(v, self.numel, "v"),
                                            _dev_ptr(u, self.nparam, "u") if self.nparam else None,
                                            _dev_ptr(phi_out, self.numel, "phi_out", True),
                                            _dev_ptr(jv_out, self.numel, "jv_out", True)), self._ctx)
        return phi_out, jv_out

    def year_adjoint(self, y0, u, ybar1, ybar0, ckpt_every=240):
        """ybar0 = phi_y^T ybar1 (into the CUDA tensor ybar0); returns ubar = phi_u^T ybar1 (numpy)."""
        self._sync_stream()
        ubar = np.zeros(max(self.nparam, 1))
        _check(self._L.metos3d_year_adjoint(self._ctx, _dev_ptr(y0, self.numel, "y0"), _dev_ptr(u, self.nparam, "u"),
                                            _dev_ptr(ybar1, self.numel, "ybar1"),
                                            _dev_ptr(ybar0, self.numel, "ybar0", True), _dp(ubar),
                                            int(ckpt_every)), self._ctx)
        return ubar[:self.nparam]

    def year_map_host(self, y0, u, out=None):
        self._sync_stream()
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        if out is None:
            out = np.empty_like(y0)
        if y0.size != self.numel or out.size != self.numel:
            raise ValueError("state must hold ntracer * n values")
        _check(self._L.metos3d_year_map_host(self._ctx, _dp(y0), _dp(out), _dp(u)), self._ctx)
        return out

    def year_map_host_ptr(self, y0_ptr, y1_ptr, u_ptr):
        """Year map on raw host pointers (e.g. pinned torch CPU tensors)."""
        self._sync_stream()
        dp = C.POINTER(C.c_double)
        _check(self._L.metos3d_year_map_host(self._ctx, C.cast(y0_ptr, dp), C.cast(y1_ptr, dp),
                                             C.cast(u_ptr, dp)), self._ctx)

    def mass(self, y):
        self._sync_stream()
        out = C.c_double()
        _check(self._L.metos3d_mass(self._ctx, _dev_ptr(y, self.numel, "y"), C.byref(out)), self._ctx)
        return out.value

    def residual(self, a, b):
        self._sync_stream()
        out = C.c_double()
        _check(self._L.metos3d_residual(self._ctx, _dev_ptr(a, self.numel, "a"), _dev_ptr(b, self.numel, "b"),
                                        C.byref(out)), self._ctx)
        return out.value

    def check_finite(self, y):
        self._sync_stream()
        return self._L.metos3d_check_finite(self._ctx, _dev_ptr(y, self.numel, "y"))

    def spinup(self, y, u, nyears, tol=0.0):
        """y <- phi(y) for up to nyears years in place; returns the residual of every year."""
        self._sync_stream()
        res = np.zeros(max(int(nyears), 1))
        done = C.c_int()
        _check(self._L.metos3d_spinup(self._ctx, _dev_ptr(y, self.numel, "y", True),
                                      _dev_ptr(u, self.nparam, "u") if self.nparam else None, int(nyears),
                                      float(tol), _dp(res), C.byref(done)), self._ctx)
        return res[:done.value]

    def newton_solve(self, y, u, check=True, **opts):
        """Newton-Krylov periodic solve in place on y; returns (status, report dict)."""
        self._sync_stream()
        o = NewtonOptions()
        self._L.metos3d_newton_default_options(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        rep = NewtonReport()
        st = self._L.metos3d_newton_solve(self._ctx, _dev_ptr(y, self.numel, "y", True),
                                          _dev_ptr(u, self.nparam, "u") if self.nparam else None,
                                          C.byref(o), C.byref(rep))
        if check and st not in (M3D_OK, M3D_NOT_CONVERGED):
            _check(st, self._ctx)
        return st, rep.to_dict()

    def periodic_gradient(self, ystar, u, g, lam=None, check=True, **opts):
        """(d ys/d u)^T g at the periodic solution ys (metos3d_periodic_gradient); lam, if given,
        receives the adjoint solution.  Returns (status, ubar ndarray, report dict)."""
        self._sync_stream()
        o = GradientOptions()
        self._L.metos3d_gradient_default_options(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        rep = GradientReport()
        ubar = np.zeros(self.nparam)
        st = self._L.metos3d_periodic_gradient(self._ctx, _dev_ptr(ystar, self.numel, "ystar"),
                                               _dev_ptr(u, self.nparam, "u"), _dev_ptr(g, self.numel, "g"),
                                               _dev_ptr(lam, self.numel, "lam", True) if lam is not None else None,
                                               _dp(ubar), C.byref(o), C.byref(rep))
        if check and st not in (M3D_OK, M3D_NOT_CONVERGED):
            _check(st, self._ctx)
        return st, ubar, rep.to_dict()

    def sync(self):
        """Wait for the stream; raises Metos3dError(M3D_ERR_TIMEOUT) if the last year map timed out."""
        _check(self._L.metos3d_sync(self._ctx), self._ctx)

    def set_option(self, option, value):
        _check(self._L.metos3d_set_option(self._ctx, int(option), int(value)), self._ctx)

    def get_option(self, option):
        return int(self._L.metos3d_get_option(self._ctx, int(option)))

    def last_launch_count(self):
        return int(self._L.metos3d_last_launch_count(self._ctx))

    def last_error(self):
        return self._L.metos3d_last_error(self._ctx).decode(errors="replace")

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._L.metos3d_free(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _year_map_function():
    """torch.autograd.Function for the year map: forward metos3d_year_map, backward the adjoint."""
    torch = _torch()

    class YearMap(torch.autograd.Function):
        @staticmethod
        def forward(fctx, y0, u, m3d_ctx, ckpt_every=240):
            y1 = torch.empty_like(y0)
            m3d_ctx.year_map(y0.detach().contiguous(), y1, u.detach().contiguous())
            fctx.save_for_backward(y0, u)
            fctx.m3d_ctx = m3d_ctx
            fctx.ckpt_every = ckpt_every
            return y1

        @staticmethod
        def backward(fctx, gy1):
            y0, u = fctx.saved_tensors
            gy0 = torch.empty_like(y0)
            ubar = fctx.m3d_ctx.year_adjoint(y0.detach().contiguous(), u.detach().contiguous(),
                                             gy1.detach().contiguous(), gy0, fctx.ckpt_every)
            gu = torch.from_numpy(ubar).to(device=u.device, dtype=u.dtype)
            return gy0, gu, None, None

    return YearMap


_YearMap = None


def year_map_autograd(y0, u, ctx, ckpt_every=240):
    """phi(y0; u) as a differentiable torch operation (gradients by the adjoint year map)."""
    global _YearMap
    if _YearMap is None:
        _YearMap = _year_map_function()
    return _YearMap.apply(y0, u, ctx, ckpt_every)


def _echeck(status, ens=None):
    if status != M3D_OK:
        msg = load().metos3d_ensemble_last_error(ens).decode(errors="replace")
        raise Metos3dError(status, msg)
    return status


class Ensemble:
    """Members -- (model id, parameters) -- advanced together on one grid (metos3d_ensemble_*).

    ``members``: a sequence of (model_id, u) pairs or of objects with ``model`` and ``u``.
    States are CUDA float64 tensors of shape (W, n): member m's tracers are rows
    ``offsets[m]:offsets[m + 1]``.  ``tangent=True`` makes a tangent ensemble
    (metos3d_ensemble_init_tangent): states of shape (2W, n), the members' states on top of
    their perturbations; ``year_map`` then returns [phi(y); phi'(y) v].
    """

    def __init__(self, *, col_start, h, zc, vol, lat, exp_rowptr, exp_colidx, exp_val, imp_blk, members,
                 nsub=1, nstep=2880, stream=None, tangent=False):
        torch = _torch()
        L = load()
        self._L = L
        cs = np.ascontiguousarray(col_start, dtype=np.int32)
        n, ncol = int(cs[-1]), int(cs.shape[0] - 1)
        h, zc, vol, lat = (np.ascontiguousarray(a, dtype=np.float64) for a in (h, zc, vol, lat))
        rp = np.ascontiguousarray(exp_rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(exp_colidx, dtype=np.int32)
        ev = np.ascontiguousarray(exp_val, dtype=np.float64)
        ib = np.ascontiguousarray(imp_blk, dtype=np.float64)
        g = _Grid(n, ncol, _ip(cs), _dp(h), _dp(zc), _dp(vol), _dp(lat))
        m = _Matrices(ev.shape[0], ci.shape[0], _ip(rp), _ip(ci), _dp(ev), ib.shape[1], _dp(ib))
        specs = [(int(getattr(x, "model", x[0] if isinstance(x, tuple) else 0)),
                  np.ascontiguousarray(getattr(x, "u", x[1] if isinstance(x, tuple) else None), dtype=np.float64))
                 for x in members]
        mem = (_Member * len(specs))()
        for i, (model, u) in enumerate(specs):
            mem[i] = _Member(model, u.shape[0], _dp(u))
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        e = C.c_void_p()
        init = L.metos3d_ensemble_init_tangent if tangent else L.metos3d_ensemble_init
        _echeck(init(C.byref(e), C.byref(g), C.byref(m), len(specs), mem, int(nsub), int(nstep),
                     C.c_void_p(stream.cuda_stream)))
        self.tangent = bool(tangent)
        self._e = e
        self.models = [mdl for mdl, _ in specs]
        self.nparams = [u.shape[0] for _, u in specs]
        nm, W, nn, G = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        offs = (C.c_int * (len(specs) + 1))()
        _echeck(L.metos3d_ensemble_layout(e, C.byref(nm), C.byref(W), C.byref(nn), C.byref(G), offs), e)
        self.nmember, self.width, self.n, self.ngroup = nm.value, W.value, nn.value, G.value
        self.offsets = [int(v) for v in offs]
        self.nstep = int(nstep)

    @classmethod
    def from_problem(cls, prob, members, **kw):
        return cls(col_start=prob.col_start, h=prob.h, zc=prob.zc, vol=prob.vol, lat=prob.lat,
                   exp_rowptr=prob.exp_rowptr, exp_colidx=prob.exp_colidx, exp_val=prob.exp_val,
                   imp_blk=prob.imp_blk, nstep=prob.nstep, members=members, **kw)

    @property
    def numel(self):
        return self.width * self.n

    def _sync_stream(self):
        torch = _torch()
        s = torch.cuda.current_stream()
        if s.cuda_stream != self._stream.cuda_stream:
            self._stream = s
            _echeck(self._L.metos3d_ensemble_set_stream(self._e, C.c_void_p(s.cuda_stream)), self._e)

    def new_state(self):
        torch = _torch()
        return torch.zeros((self.width, self.n), dtype=torch.float64, device="cuda")

    def member(self, Y, m):
        """Rows of member m in an ensemble state."""
        return Y[self.offsets[m]:self.offsets[m + 1]]

    def steps(self, j0, nsteps, Y0, Y1):
        self._sync_stream()
        _echeck(self._L.metos3d_ensemble_steps(self._e, int(j0), int(nsteps), _dev_ptr(Y0, self.numel, "Y0"),
                                               _dev_ptr(Y1, self.numel, "Y1", True)), self._e)
        return Y1

    def year_map(self, Y0, Y1):
        self._sync_stream()
        _echeck(self._L.metos3d_ensemble_year_map(self._e, _dev_ptr(Y0, self.numel, "Y0"),
                                                  _dev_ptr(Y1, self.numel, "Y1", True)), self._e)
        return Y1

    def year_adjoint(self, Y0, Ybar1, Ybar0, ckpt_every=240):
        """Reverse sweep of every member's year map (metos3d_ensemble_year_adjoint): Ybar0 receives
        phi_y^T Ybar1; returns the list of the members' parameter gradients phi_u^T Ybar1."""
        self._sync_stream()
        ub = np.zeros(sum(self.nparams))
        _echeck(self._L.metos3d_ensemble_year_adjoint(self._e, _dev_ptr(Y0, self.numel, "Y0"),
                                                      _dev_ptr(Ybar1, self.numel, "Ybar1"),
                                                      _dev_ptr(Ybar0, self.numel, "Ybar0", True), _dp(ub),
                                                      int(ckpt_every)), self._e)
        out, at = [], 0
        for k in self.nparams:
            out.append(ub[at:at + k].copy())
            at += k
        return out

    def newton_solve(self, Y, vol, tangent_ensemble=None, **opts):
        """Periodic solve of every member in place on Y (metos3d_ensemble_newton_solve), with
        tangent products from ``tangent_ensemble`` (jv=JV_TANGENT) or finite differences;
        returns (status, list of the members' report dicts)."""
        self._sync_stream()
        o = NewtonOptions()
        self._L.metos3d_newton_default_options(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        reps = (NewtonReport * self.nmember)()
        vol = np.ascontiguousarray(vol, dtype=np.float64)
        st = self._L.metos3d_ensemble_newton_solve(self._e, tangent_ensemble._e if tangent_ensemble else None,
                                                   _dev_ptr(Y, self.numel, "Y", True), _dp(vol), C.byref(o), reps)
        if st not in (M3D_OK, M3D_NOT_CONVERGED):
            raise Metos3dError(st, "metos3d_ensemble_newton_solve failed")
        return st, [r.to_dict() for r in reps]

    def set_params(self, m, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape[0] != self.nparams[m]:
            raise ValueError("member %d takes %d parameters" % (m, self.nparams[m]))
        _echeck(self._L.metos3d_ensemble_set_params(self._e, int(m), _dp(u)), self._e)

    def set_tiling(self, cols_per_block, warps_per_block):
        _echeck(self._L.metos3d_ensemble_set_tiling(self._e, int(cols_per_block), int(warps_per_block)), self._e)

    def get_tiling(self):
        a, b = C.c_int(), C.c_int()
        _echeck(self._L.metos3d_ensemble_get_tiling(self._e, C.byref(a), C.byref(b)), self._e)
        return a.value, b.value

    def autotune(self, Y, nsteps=10):
        """Time the candidate tilings from state Y, keep the fastest; (cols, warps, ms per step)."""
        self._sync_stream()
        a, b, ms = C.c_int(), C.c_int(), C.c_double()
        _echeck(self._L.metos3d_ensemble_autotune(self._e, _dev_ptr(Y, self.numel, "Y"), int(nsteps), C.byref(a),
                                                  C.byref(b), C.byref(ms)), self._e)
        return a.value, b.value, ms.value

    def last_launch_count(self):
        return int(self._L.metos3d_ensemble_last_launch_count(self._e))

    def close(self):
        if getattr(self, "_e", None):
            self._L.metos3d_ensemble_free(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
