"""Gradient at the periodic solution on the CPU oracle -- TEST INFRASTRUCTURE ONLY.

The parameter optimisation the paper motivates (Sections 1 and 9) fits the model to data
through its periodic state ys(u), the fixed point ys = phi(ys; u) that Newton's method
finds (Sections 6 and 7).  phi conserves the total mass sum_i vol_i y_i, so for each mass
there is one periodic state; the derivative of ys with respect to u at fixed mass is the
solution dY (one column per parameter) of

    (I - phi_y) dY = phi_u,    w^T dY = 0,    w = vol repeated per tracer,

the implicit function theorem applied to y - phi(y; u) = 0 restricted to one mass.  The
gradient of a misfit J(ys(u)) is then dY^T g with g = dJ/dy at ys.

This module states that definition literally for small grids: it forms phi_y and phi_u row
by row from the oracle's adjoint year map (row i of both is the adjoint applied to the unit
vector e_i), stacks the mass condition under I - phi_y, and solves the consistent
(N+1) x N system by least squares.  No Krylov method, no projection trick: a dense solve a
reader can check against the equations above.
"""
from __future__ import annotations

import numpy as np

from . import MODEL_NDOP, year_adjoint


def year_jacobians(P, y, u, model=MODEL_NDOP, nsub=1):
    """(phi_y, phi_u) of the year map at (y, u) as dense arrays [N][N] and [N][nparam], N the
    number of state entries, from one adjoint year map per row."""
    y = np.asarray(y, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    N = y.size
    Jy = np.empty((N, N))
    Ju = np.empty((N, u.size))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        ybar0, ubar = year_adjoint(P, y, u, e.reshape(y.shape), model=model, nsub=nsub)
        Jy[i] = ybar0.ravel()
        Ju[i] = ubar
    return Jy, Ju


def periodic_state_derivative(P, ystar, u, model=MODEL_NDOP, nsub=1):
    """dY = d ys / d u at fixed mass, [N][nparam]: the least-squares solution of the stacked
    system [I - phi_y; w^T] dY = [phi_u; 0], which is consistent (w^T phi_y = w^T and
    w^T phi_u = 0 because phi conserves mass), so its residual is zero up to rounding."""
    ystar = np.asarray(ystar, dtype=np.float64)
    Jy, Ju = year_jacobians(P, ystar, u, model=model, nsub=nsub)
    N = ystar.size
    w = np.tile(np.asarray(P.prob.vol, dtype=np.float64), ystar.shape[0])
    w = w / np.linalg.norm(w)         # the condition w^T dY = 0 does not depend on w's scale
    A = np.vstack([np.eye(N) - Jy, w[None, :]])
    rhs = np.vstack([Ju, np.zeros((1, Ju.shape[1]))])
    dY, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return dY


def periodic_gradient(P, ystar, u, g, model=MODEL_NDOP, nsub=1):
    """(d ys / d u)^T g at the periodic state ys; g = dJ/dy at ys, shaped like ys."""
    dY = periodic_state_derivative(P, ystar, u, model=model, nsub=nsub)
    return dY.T @ np.asarray(g, dtype=np.float64).ravel()
