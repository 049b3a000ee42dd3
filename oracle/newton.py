"""Spin-up and Newton-Krylov periodic solve on the CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain statement of the solvers the paper compares (Sections 4, 6 and 7):

* spin-up: the fixed-point iteration y <- phi(y), one model year at a time, recording the
  residual ||y - phi(y)||_2 after every year;
* Newton's method on F(y) = y - phi(y) = 0, globalised by a backtracking line search with
  cubic interpolation, each Newton system (I - phi'(y)) s = -F(y) solved inexactly by
  restarted GMRES with modified Gram-Schmidt orthogonalisation, Jacobian-vector products
  by finite differences, and the Eisenstat-Walker choice of the inner tolerances.

The year map comes from the C oracle; everything else is numpy, written for reading.
Parameters not given by the paper (line-search constants, forcing-term constants, finite
difference step) are the textbook values named in each function.
"""
from __future__ import annotations

import math

import numpy as np

from . import MODEL_NDOP, year_map


def spinup(P, y0, u, nyears, model=MODEL_NDOP, nsub=1, tol=0.0):
    """y <- phi(y) for up to nyears years; returns (y, residual history)."""
    y = np.array(y0, dtype=np.float64)
    hist = []
    for _ in range(nyears):
        py = year_map(P, y, u, model=model, nsub=nsub)
        r = float(np.linalg.norm((py - y).ravel()))
        hist.append(r)
        y = py
        if r <= tol:
            break
    return y, hist


def gmres_mgs(apply_J, b, tol_rel, restart, maxit):
    """Restarted GMRES for J x = b from x = 0, modified Gram-Schmidt, Givens rotations.

    Stops when ||b - J x|| <= tol_rel ||b|| or after maxit iterations.
    Returns (x, iterations, final relative residual estimate).
    """
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b.copy()
    beta = bnorm
    while True:
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        V[0] = r / beta
        g[0] = beta
        k_used = 0
        for k in range(restart):
            w = apply_J(V[k])
            for i in range(k + 1):                      # modified Gram-Schmidt
                H[i, k] = float(np.dot(w, V[i]))
                w = w - H[i, k] * V[i]
            H[k + 1, k] = float(np.linalg.norm(w))
            if H[k + 1, k] > 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):                          # previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            d = math.hypot(H[k, k], H[k + 1, k])        # new rotation
            cs[k], sn[k] = (1.0, 0.0) if d == 0.0 else (H[k, k] / d, H[k + 1, k] / d)
            H[k, k] = d
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            if abs(g[k + 1]) <= tol_rel * bnorm or it >= maxit:
                break
        yk = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used]) if k_used else np.zeros(0)
        x = x + V[:k_used].T @ yk
        res = abs(g[k_used])
        if res <= tol_rel * bnorm or it >= maxit:
            return x, it, res / bnorm
        r = b - apply_J(x)
        beta = float(np.linalg.norm(r))
        if beta <= tol_rel * bnorm:
            return x, it, beta / bnorm


GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0


def forcing_term(r, r_prev, eta_prev, tol, eta0=0.3, gamma=0.9, alpha=GOLDEN, eta_max=0.9):
    """Inner tolerance of the next Newton step (Eisenstat & Walker 1996, choice 2).

    First step: eta_0.  Later steps: gamma (||F_k|| / ||F_{k-1}||)^alpha, raised to the
    safeguard gamma eta_{k-1}^alpha when the safeguard exceeds 0.1 (so that eta does not
    drop sharply after one lucky step).  Finally kept within [0.5 tol / ||F_k||, eta_max]:
    no oversolving of the last step and never a useless tolerance near 1.
    """
    if eta_prev is None:
        eta = eta0
    else:
        eta = gamma * (r / r_prev) ** alpha
        safe = gamma * eta_prev ** alpha
        if safe > 0.1:
            eta = max(eta, safe)
    return min(max(eta, 0.5 * tol / r), eta_max)


def quadratic_backtrack(f0, slope, lam, f_lam):
    """Minimiser of the quadratic model m(x) = f0 + slope x + c x^2 fitted to m(lam) = f_lam
    (Dennis & Schnabel, Section 6.3.2: the first backtrack)."""
    return -slope * lam * lam / (2.0 * (f_lam - f0 - slope * lam))


def cubic_backtrack(f0, slope, lam, f_lam, lam_prev, f_prev):
    """Local minimiser of the cubic model m(x) = f0 + slope x + b x^2 + a x^3 fitted to the last
    two trials, m(lam) = f_lam and m(lam_prev) = f_prev (Dennis & Schnabel, Section 6.3.2: every
    later backtrack).  m'(x) = slope + 2 b x + 3 a x^2 = 0 at x = (-b + sqrt(b^2 - 3 a slope)) / (3 a);
    with a = 0 the model is the quadratic and x = -slope / (2 b)."""
    r1 = f_lam - f0 - lam * slope
    r2 = f_prev - f0 - lam_prev * slope
    den = lam - lam_prev
    a = (r1 / (lam * lam) - r2 / (lam_prev * lam_prev)) / den
    b = (-lam_prev * r1 / (lam * lam) + lam * r2 / (lam_prev * lam_prev)) / den
    if a == 0.0:
        return -slope / (2.0 * b)
    disc = max(b * b - 3.0 * a * slope, 0.0)
    return (-b + math.sqrt(disc)) / (3.0 * a)


def line_search(f, f0, slope, armijo=1e-4, lam_min=1e-4, lo=0.1, hi=0.5):
    """Backtracking line search along a descent direction of f, with f(0) = f0, f'(0) = slope < 0
    (Dennis & Schnabel, Algorithm A6.3.1).

    Tries lam = 1 first and accepts the first lam with the Armijo decrease
    f(lam) <= f0 + armijo lam slope.  After a failed trial the next lam is the minimiser of the
    quadratic model (first backtrack) or of the cubic model through the last two trials (later
    backtracks), kept within [lo, hi] times the failed lam.  A trial whose f is not finite (the
    model state left its domain) gives no model: the next lam is lo times it, and the next
    finite failure starts from the quadratic model again.  A lam below lam_min is not tried:
    the search fails and returns (0.0, f0, trials), no step.
    Returns (lam, f(lam), trials), trials the list of (lam, f(lam)) in the order tried.
    """
    lam, prev, trials = 1.0, None, []
    while lam >= lam_min:
        fl = f(lam)
        trials.append((lam, fl))
        if not math.isfinite(fl):
            prev = None
            lam = lo * lam
            continue
        if fl <= f0 + armijo * lam * slope:
            return lam, fl, trials
        if prev is None:
            lt = quadratic_backtrack(f0, slope, lam, fl)
        else:
            lt = cubic_backtrack(f0, slope, lam, fl, prev[0], prev[1])
        prev = (lam, fl)
        lam = min(max(lt, lo * lam), hi * lam) if math.isfinite(lt) else lo * lam
    return 0.0, f0, trials


def newton_krylov(P, y0, u, tol=1e-8, max_newton=40, restart=200, max_krylov=200, fd_eps=1e-8,
                  model=MODEL_NDOP, nsub=1, jv=None, record_steps=False):
    """Newton-Krylov periodic solve of the year map of P; returns (y, report dict).

    phi conserves sum_i vol_i y_i, so I - phi'(y) is singular and the periodic solution is
    unique only for a given total mass: the Newton steps are projected on the zero-mass
    directions (w = vol repeated per tracer), see newton_solve.
    """
    shape = np.shape(y0)
    wmass = np.tile(np.asarray(P.prob.vol, dtype=np.float64), shape[0])

    def phi(v):
        return year_map(P, v.reshape(shape), u, model=model, nsub=nsub).ravel()

    jvf = None
    if jv is not None:
        def jvf(y, py, v):
            return jv(y.reshape(shape), py.reshape(shape), v.reshape(shape)).ravel()
    y, rep = newton_solve(phi, np.asarray(y0, dtype=np.float64).ravel(), tol=tol, max_newton=max_newton,
                          restart=restart, max_krylov=max_krylov, fd_eps=fd_eps, jv=jvf, wmass=wmass,
                          record_steps=record_steps)
    return y.reshape(shape), rep


def newton_solve(phi, y0, tol=1e-8, max_newton=40, restart=200, max_krylov=200, fd_eps=1e-8, jv=None,
                 wmass=None, record_steps=False):
    """Newton's method on F(y) = y - phi(y) = 0 for a map phi of flat vectors; returns (y, report).

    Forcing terms: forcing_term (Eisenstat & Walker, choice 2); each Newton system
    (I - phi'(y)) s = -F(y) solved by gmres_mgs to that tolerance.  Jacobian-vector products:
    J v = v - (phi(y + h v) - phi(y)) / h, h = fd_eps ||y|| / ||v||, unless a function
    jv(y, phi_y, v) returning phi'(y) v is given.  wmass (optional): every step s is projected
    on the directions orthogonal to it, s <- s - (w.s / w.w) w (for the year map, w = vol
    repeated per tracer: the mass it conserves; the projection removes the rounding drift of
    the finite-difference products).  Line search: line_search on f(lam) = ||F(y + lam s)||^2 / 2,
    whose slope at 0 is F^T J s.  GMRES's step s minimises ||F + J s|| over its Krylov space,
    so its residual rho = ||F + J s|| is orthogonal to J s and F^T J s = -(||F||^2 - rho^2) (in one
    GMRES cycle, which restart >= max_krylov gives): the inexact step's own slope, not the
    -||F||^2 of an exact Newton step (with eta up to 0.9 the two differ by a factor up to 5).
    The report holds, per Newton step, eta, the GMRES iterations and residual rho, the slope,
    the accepted lam (0 where the line search found no acceptable step: the solve then stops at
    the current iterate with line_search_failed) and every lam tried; with record_steps, also the steps s and the states
    y they start from.
    """
    y = np.array(y0, dtype=np.float64)
    py = phi(y)
    F = y - py
    r = float(np.linalg.norm(F))
    rep = {"residuals": [r], "krylov": [], "year_maps": 1, "lambdas": [], "etas": [], "slopes": [],
           "gmres_residuals": [], "trials": [], "converged": False, "line_search_failed": False}
    if not math.isfinite(r):
        return y, rep
    if record_steps:
        rep["steps"], rep["states"] = [], []
    eta_prev, r_prev = None, None
    for _ in range(max_newton):
        if r <= tol:
            rep["converged"] = True
            break
        eta = forcing_term(r, r_prev, eta_prev, tol)
        ynorm = float(np.linalg.norm(y))

        def apply_J(v):
            if jv is not None:
                return v - jv(y, py, v)
            h = fd_eps * ynorm / float(np.linalg.norm(v))
            rep["year_maps"] += 1
            return v - (phi(y + h * v) - py) / h

        nfd = rep["year_maps"]
        s, its, res_rel = gmres_mgs(apply_J, -F, eta, restart, max_krylov)
        if wmass is not None:
            s = s - (float(np.dot(wmass, s)) / float(np.dot(wmass, wmass))) * wmass
        if jv is not None:
            rep["year_maps"] = nfd + 2 * its         # a tangent year map costs about two
        rho = res_rel * r
        slope = -(r * r - rho * rho)
        cache = {}

        def f(lam):
            cache[lam] = phi(y + lam * s)
            rep["year_maps"] += 1
            Fl = y + lam * s - cache[lam]
            return 0.5 * float(np.dot(Fl, Fl))

        lam, fn, trials = line_search(f, 0.5 * r * r, slope)
        if record_steps:
            rep["steps"].append(s.copy())
            rep["states"].append(y.copy())
        rep["krylov"].append(its)
        rep["etas"].append(eta)
        rep["gmres_residuals"].append(rho)
        rep["slopes"].append(slope)
        rep["lambdas"].append(lam)
        rep["trials"].append([t[0] for t in trials])
        if lam == 0.0:
            # no acceptable step along s: stop at the current iterate
            rep["line_search_failed"] = True
            rep["residuals"].append(r)
            break
        yn = y + lam * s
        pyn = cache[lam]
        y, py, F = yn, pyn, yn - pyn
        r_prev, eta_prev = r, eta
        r = math.sqrt(2.0 * fn)
        rep["residuals"].append(r)
    rep["converged"] = r <= tol
    return y, rep
