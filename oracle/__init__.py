"""CPU oracle of the TMM year map -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C implementation (``tmm_oracle.c``) of the Metos3D time step, year map and
biogeochemical models (arXiv:1410.0204, Sections 2.2, 3, 4, 5: PO4-DOP, PO4-DOP-PHY, and the
N and NPZD-DOP models of the batched ensemble), loaded here through ctypes.  The ensemble
year map is each member's own year map: the members share the transport and nothing else.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library under
``paper_1410_0204_gb300/``; both read their inputs from ``m3d_inputs``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MODEL_NONE = 0
MODEL_N = 1
MODEL_NDOP = 2
MODEL_PHY = 3
MODEL_NPZD = 5

_lib = None


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("ncol", C.c_int), ("nnz", C.c_int), ("nmonth", C.c_int), ("nstep", C.c_int),
        ("col_start", C.POINTER(C.c_int)), ("h", C.POINTER(C.c_double)), ("zc", C.POINTER(C.c_double)),
        ("lat", C.POINTER(C.c_double)), ("rowptr", C.POINTER(C.c_int)), ("colidx", C.POINTER(C.c_int)),
        ("exp_val", C.POINTER(C.c_double)), ("blk_off", C.POINTER(C.c_longlong)),
        ("imp_blk", C.POINTER(C.c_double)), ("s_imp", C.c_longlong),
    ]


def lib():
    global _lib
    if _lib is None:
        # M3D_ORACLE_LIB lets the mutation check load a deliberately broken copy
        path = os.environ.get("M3D_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.oracle_month_weights.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
        L.oracle_insolation.argtypes = [C.c_double, C.c_double, dp]
        L.oracle_insolation.restype = C.c_double
        L.oracle_bgc.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp,
                                 C.c_int, dp, C.c_int]
        L.oracle_step.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int, dp]
        L.oracle_year_map.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int]
        L.oracle_steps.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int]
        L.oracle_bgc_tangent.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp,
                                         C.c_int, dp, C.c_int]
        L.oracle_year_tangent.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, dp, dp, dp, dp, dp, C.c_int, C.c_int]
        L.oracle_bgc_adjoint.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, dp, dp, dp,
                                         dp, dp, C.c_int, dp, dp, C.c_int]
        L.oracle_year_adjoint.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, dp, dp, dp]
        L.oracle_set_threads.argtypes = [C.c_int]
        # one thread unless asked otherwise: the oracle's reference mode is single-threaded
        L.oracle_set_threads(int(os.environ.get("M3D_ORACLE_THREADS", "1")))
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """ctypes view of an ``m3d_inputs.Problem``; keeps the arrays alive."""

    def __init__(self, prob):
        self.prob = prob
        self._keep = dict(
            col_start=np.ascontiguousarray(prob.col_start, dtype=np.int32),
            h=_f64(prob.h), zc=_f64(prob.zc), lat=_f64(prob.lat),
            rowptr=np.ascontiguousarray(prob.exp_rowptr, dtype=np.int32),
            colidx=np.ascontiguousarray(prob.exp_colidx, dtype=np.int32),
            exp_val=_f64(prob.exp_val), blk_off=np.ascontiguousarray(prob.blk_off, dtype=np.int64),
            imp_blk=_f64(prob.imp_blk))
        k = self._keep
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        self.s = _Problem(prob.n, prob.ncol, prob.nnz, prob.nmonth, prob.nstep,
                          ip(k["col_start"]), _dp(k["h"]), _dp(k["zc"]), _dp(k["lat"]),
                          ip(k["rowptr"]), ip(k["colidx"]), _dp(k["exp_val"]),
                          k["blk_off"].ctypes.data_as(C.POINTER(C.c_longlong)), _dp(k["imp_blk"]),
                          int(prob.s_imp))


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the oracle loops; returns the count in effect."""
    return int(lib().oracle_set_threads(int(n)))


def month_weights(j: int, nstep: int = 2880, nmonth: int = 12):
    m0, m1, w = C.c_int(), C.c_int(), C.c_double()
    lib().oracle_month_weights(j, nstep, nmonth, C.byref(m0), C.byref(m1), C.byref(w))
    return m0.value, m1.value, w.value


def insolation(lat_deg: float, t: float):
    """Daily-mean top-of-atmosphere insolation [W/m^2] and daylight fraction."""
    df = C.c_double()
    q = lib().oracle_insolation(float(lat_deg), float(t), C.byref(df))
    return q, df.value


def bgc(y, h, d, u, t=0.0, dt=1.0 / 2880, lat=0.0, insol=0.0, dayfrac=0.5, ice=0.0,
        model=MODEL_NDOP, nsub=1):
    """The model interface of Section 5.2 on one column; y is (ntracer, nlayer). Returns ybgc."""
    y = _f64(y)
    ntr, nl = y.shape
    h, d, u = _f64(h), _f64(d), _f64(u)
    out = np.zeros_like(y)
    zeros = np.zeros(nl)
    rc = lib().oracle_bgc(model, t, dt, lat, insol, dayfrac, ice, 0.0, ntr, nl, _dp(h), _dp(d),
                          _dp(zeros), _dp(zeros), _dp(y), _dp(out), u.shape[0], _dp(u), nsub)
    if rc != 0:
        raise ValueError("oracle_bgc rejected its arguments")
    return out


def step(P: Problem, j: int, y, u, model=MODEL_NDOP, nsub=1):
    y = _f64(y)
    u = _f64(u)
    out = np.empty_like(y)
    work = np.empty_like(y)
    rc = lib().oracle_step(C.byref(P.s), model, y.shape[0], j, _dp(y), _dp(out), _dp(u), u.shape[0], nsub, _dp(work))
    if rc != 0:
        raise ValueError("oracle_step failed")
    return out


def steps(P: Problem, j0: int, nsteps: int, y, u, model=MODEL_NDOP, nsub=1):
    y = _f64(y)
    u = _f64(u)
    out = np.empty_like(y)
    rc = lib().oracle_steps(C.byref(P.s), model, y.shape[0], j0, nsteps, _dp(y), _dp(out), _dp(u), u.shape[0], nsub)
    if rc != 0:
        raise ValueError("oracle_steps failed")
    return out


def year_map(P: Problem, y0, u, model=MODEL_NDOP, nsub=1):
    y0 = _f64(y0)
    u = _f64(u)
    out = np.empty_like(y0)
    rc = lib().oracle_year_map(C.byref(P.s), model, y0.shape[0], _dp(y0), _dp(out), _dp(u), u.shape[0], nsub)
    if rc != 0:
        raise ValueError("oracle_year_map failed")
    return out


def bgc_tangent(y, dy, h, d, u, t=0.0, dt=1.0 / 2880, lat=0.0, insol=0.0, dayfrac=0.5, ice=0.0,
                model=MODEL_NDOP, nsub=1):
    """The model interface and its tangent along dy on one column; returns (ybgc, dybgc)."""
    y = _f64(y)
    dy = _f64(dy)
    ntr, nl = y.shape
    h, d, u = _f64(h), _f64(d), _f64(u)
    out = np.zeros_like(y)
    dout = np.zeros_like(y)
    rc = lib().oracle_bgc_tangent(model, t, dt, lat, insol, dayfrac, ice, 0.0, ntr, nl, _dp(h), _dp(d),
                                  _dp(y), _dp(dy), _dp(out), _dp(dout), u.shape[0], _dp(u), nsub)
    if rc != 0:
        raise ValueError("oracle_bgc_tangent rejected its arguments")
    return out, dout


def year_tangent(P: Problem, y0, v, u, model=MODEL_NDOP, nsub=1):
    """(phi(y0), phi'(y0) v)."""
    y0 = _f64(y0)
    v = _f64(v)
    u = _f64(u)
    y1 = np.empty_like(y0)
    jv = np.empty_like(y0)
    rc = lib().oracle_year_tangent(C.byref(P.s), model, y0.shape[0], _dp(y0), _dp(v), _dp(y1), _dp(jv), _dp(u),
                                   u.shape[0], nsub)
    if rc != 0:
        raise ValueError("oracle_year_tangent failed")
    return y1, jv


def bgc_adjoint(y, ybgc_bar, h, d, u, dt=1.0 / 2880, insol=0.0, ice=0.0, model=MODEL_NDOP, nsub=1):
    """Reverse of the model interface: returns (ybar, ubar) for the cotangent ybgc_bar."""
    y = _f64(y)
    yb_in = _f64(ybgc_bar)
    ntr, nl = y.shape
    h, d, u = _f64(h), _f64(d), _f64(u)
    ybar = np.zeros_like(y)
    ubar = np.zeros(u.shape[0])
    rc = lib().oracle_bgc_adjoint(model, dt, insol, ice, ntr, nl, _dp(h), _dp(d), _dp(y), _dp(yb_in), _dp(ybar),
                                  u.shape[0], _dp(u), _dp(ubar), nsub)
    if rc != 0:
        raise ValueError("oracle_bgc_adjoint rejected its arguments")
    return ybar, ubar


def year_adjoint(P: Problem, y0, u, ybar1, model=MODEL_NDOP, nsub=1):
    """(phi_y^T ybar1, phi_u^T ybar1) for y1 = phi(y0; u)."""
    y0 = _f64(y0)
    u = _f64(u)
    yb1 = _f64(ybar1)
    ybar0 = np.empty_like(y0)
    ubar = np.zeros(u.shape[0])
    rc = lib().oracle_year_adjoint(C.byref(P.s), model, y0.shape[0], _dp(y0), _dp(u), u.shape[0], nsub, _dp(yb1),
                                   _dp(ybar0), _dp(ubar))
    if rc != 0:
        raise ValueError("oracle_year_adjoint failed")
    return ybar0, ubar


def ensemble_steps(P: Problem, j0: int, nsteps: int, states, members, nsub=1):
    """nsteps TMM steps of every member (a list of [ntracer][n] states), each on its own."""
    return [steps(P, j0, nsteps, y, m.u, model=m.model, nsub=nsub) for y, m in zip(states, members)]


def ensemble_year_map(P: Problem, states, members, nsub=1):
    """The year map of every member of an ensemble (members are independent)."""
    return [year_map(P, y, m.u, model=m.model, nsub=nsub) for y, m in zip(states, members)]
