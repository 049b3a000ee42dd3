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


def newton_krylov(P, y0, u, tol=1e-8, max_newton=40, restart=200, max_krylov=200, fd_eps=1e-8,
                  model=MODEL_NDOP, nsub=1, jv=None):
    """Newton-Krylov periodic solve; returns (y, report dict).

    Forcing terms (Eisenstat & Walker, choice 2): eta_0 = 0.3, then
    eta_k = 0.9 (||F_k|| / ||F_{k-1}||)^((1+sqrt 5)/2), safeguarded by 0.9 eta_{k-1}^((1+sqrt 5)/2)
    when that exceeds 0.1, and kept in [0.5 tol / ||F_k||, 0.9].
    Jacobian-vector products: J v = v - (phi(y + h v) - phi(y)) / h, h = fd_eps ||y|| / ||v||,
    unless a function jv(y, phi_y, v) returning phi'(y) v is given.
    Line search: Armijo condition f(y + l s) <= f(y) + 1e-4 l f'(0) on f = ||F||^2 / 2 with
    f'(0) = -||F||^2, starting at l = 1, then quadratic and cubic backtracking with
    l in [0.1 l_prev, 0.5 l_prev] (Dennis & Schnabel).
    Mass: phi conserves sum_i vol_i y_i, so I - phi'(y) is singular and the periodic
    solution is unique only for a given total mass.  Every Newton step s is projected onto
    the zero-mass directions, s <- s - (w.s / w.w) w with w = vol repeated per tracer,
    which removes the rounding drift of the finite-difference products.
    """
    shape = np.shape(y0)
    y = np.array(y0, dtype=np.float64).ravel()
    wmass = np.tile(np.asarray(P.prob.vol, dtype=np.float64), shape[0])

    def phi(v):
        return year_map(P, v.reshape(shape), u, model=model, nsub=nsub).ravel()

    py = phi(y)
    F = y - py
    r = float(np.linalg.norm(F))
    rep = {"residuals": [r], "krylov": [], "year_maps": 1, "lambdas": [], "converged": False}
    gamma, alpha = 0.9, (1.0 + math.sqrt(5.0)) / 2.0
    eta_prev, r_prev = None, None
    for _ in range(max_newton):
        if r <= tol:
            rep["converged"] = True
            break
        if eta_prev is None:
            eta = 0.3
        else:
            eta = gamma * (r / r_prev) ** alpha
            safe = gamma * eta_prev ** alpha
            if safe > 0.1:
                eta = max(eta, safe)
        eta = min(max(eta, 0.5 * tol / r), 0.9)
        ynorm = float(np.linalg.norm(y))

        def apply_J(v):
            if jv is not None:
                return v - jv(y.reshape(shape), py.reshape(shape), v.reshape(shape)).ravel()
            h = fd_eps * ynorm / float(np.linalg.norm(v))
            rep["year_maps"] += 1
            return v - (phi(y + h * v) - py) / h

        nfd = rep["year_maps"]
        s, its, _ = gmres_mgs(apply_J, -F, eta, restart, max_krylov)
        s = s - (float(np.dot(wmass, s)) / float(np.dot(wmass, wmass))) * wmass
        rep["krylov"].append(its)
        if jv is not None:
            rep["year_maps"] = nfd + 2 * its         # a tangent year map costs about two
        f0 = 0.5 * r * r
        slope = -r * r
        lam, lam_prev, f_prev = 1.0, None, None
        while True:
            yn = y + lam * s
            pyn = phi(yn)
            rep["year_maps"] += 1
            Fn = yn - pyn
            fn = 0.5 * float(np.dot(Fn, Fn))
            if fn <= f0 + 1e-4 * lam * slope or lam < 1e-4:
                break
            if lam_prev is None:
                lt = -slope / (2.0 * (fn - f0 - slope))
            else:
                a1 = fn - f0 - lam * slope
                a2 = f_prev - f0 - lam_prev * slope
                den = lam - lam_prev
                a = (a1 / (lam * lam) - a2 / (lam_prev * lam_prev)) / den
                b = (-lam_prev * a1 / (lam * lam) + lam * a2 / (lam_prev * lam_prev)) / den
                if a == 0.0:
                    lt = -slope / (2.0 * b)
                else:
                    disc = max(b * b - 3.0 * a * slope, 0.0)
                    lt = (-b + math.sqrt(disc)) / (3.0 * a)
            lam_prev, f_prev = lam, fn
            lam = min(max(lt, 0.1 * lam), 0.5 * lam)
        rep["lambdas"].append(lam)
        y, py, F = yn, pyn, Fn
        r_prev, eta_prev = r, eta
        r = math.sqrt(2.0 * fn)
        rep["residuals"].append(r)
    rep["converged"] = r <= tol
    return y.reshape(shape), rep
