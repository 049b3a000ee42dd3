"""Pins of the oracle's gradient at the periodic solution (oracle/implicit.py).

The implicit-function derivative d ys / d u at fixed mass, and the misfit gradient built
from it, are checked against central differences of periodic states that the oracle's own
Newton-Krylov solve finds at u + h e_k and u - h e_k from the same mass, on a tiny grid.
Nothing here shares the dense solve: the differences only run the year map, its tangent (for
Newton's Jacobian-vector products) and the Newton iteration.
"""
import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from oracle import implicit
from oracle.newton import newton_krylov

NEWTON_TOL = 3e-12           # the year map's rounding floor on this grid is about 1.2e-12


@pytest.fixture(scope="module")
def setup():
    p = mi.make_problem("tiny_6x4x4")      # four layers: every parameter acts
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y0 = mi.initial_state(p)

    cache = {}

    def solve(uu, start):
        key = (tuple(uu), id(start))
        if key not in cache:
            jv = lambda y, py, v: oracle.year_tangent(P, y, v, uu)[1]
            ys, rep = newton_krylov(P, start, uu, tol=NEWTON_TOL, jv=jv, max_newton=60)
            assert rep["converged"], rep["residuals"][-3:]
            cache[key] = ys
        return cache[key].copy()

    ystar = solve(u, y0)
    return p, P, u, ystar, solve


def richardson(f, u, k, rel=1e-3):
    """Derivative of f along parameter k: central differences at h and h/2 combined so that
    their h^2 terms cancel, (4 D(h/2) - D(h)) / 3.  h is kept large against the solves'
    3e-12 residual, which divided by h is the noise of a difference."""
    def central(h):
        up, um = u.copy(), u.copy()
        up[k] += h
        um[k] -= h
        return (f(up) - f(um)) / (2 * h)
    h = rel * abs(u[k])
    return (4.0 * central(h / 2) - central(h)) / 3.0


def test_periodic_state_is_a_fixed_point_of_the_same_mass(setup):
    p, P, u, ystar, _ = setup
    assert np.linalg.norm(oracle.year_map(P, ystar, u) - ystar) <= 10 * NEWTON_TOL
    m0 = float((mi.initial_state(p).sum(axis=0) * p.vol).sum())
    assert abs(float((ystar.sum(axis=0) * p.vol).sum()) - m0) <= 1e-13 * m0


def test_state_derivative_matches_central_differences_of_newton_solves(setup):
    p, P, u, ystar, solve = setup
    dY = implicit.periodic_state_derivative(P, ystar, u)
    w = np.tile(p.vol, ystar.shape[0])
    assert np.max(np.abs(w @ dY)) <= 1e-12 * np.linalg.norm(w) * np.linalg.norm(dY)    # zero mass change
    for k in range(u.size):
        fd = richardson(lambda uu: solve(uu, ystar).ravel(), u, k)
        scale = np.max(np.abs(fd))
        assert scale > 1e-6 * np.max(np.abs(ystar)), k
        assert np.max(np.abs(dY[:, k] - fd)) <= 1e-5 * scale, (k, np.max(np.abs(dY[:, k] - fd)) / scale)


def test_misfit_gradient_matches_central_differences(setup):
    p, P, u, ystar, solve = setup
    r = mi.rng(1410, "observations")
    mask = (r.random(ystar.shape) < 0.5).astype(np.float64)
    obs = ystar * (1.0 + 0.05 * r.standard_normal(ystar.shape))

    def J(y):
        return 0.5 * float(np.sum(mask * (y - obs) ** 2))

    g = mask * (ystar - obs)
    grad = implicit.periodic_gradient(P, ystar, u, g)
    # errors of the differences scale with the terms of sum_i dY_ik g_i before they cancel
    dY = implicit.periodic_state_derivative(P, ystar, u)
    terms = np.abs(dY * g.ravel()[:, None]).sum(axis=0)
    assert np.allclose(grad, dY.T @ g.ravel(), rtol=1e-14, atol=0.0)
    for k in range(u.size):
        fd = richardson(lambda uu: J(solve(uu, ystar)), u, k)
        assert abs(grad[k] - fd) <= 1e-5 * terms[k], (k, grad[k], fd, terms[k])


def test_without_the_mass_condition_the_derivative_is_wrong(setup):
    # I - phi_y alone is singular (phi conserves mass); its minimum-norm solution differs from
    # the fixed-mass derivative, which the differences above single out
    p, P, u, ystar, solve = setup
    Jy, Ju = implicit.year_jacobians(P, ystar, u)
    N = ystar.size
    sv = np.linalg.svd(np.eye(N) - Jy, compute_uv=False)
    assert sv[-1] <= 1e-10 * sv[0]                  # singular: one zero singular value
    assert sv[-2] >= 1e-6 * sv[0]                   # and only one
    dY_free = np.linalg.lstsq(np.eye(N) - Jy, Ju, rcond=1e-10)[0]
    dY = implicit.periodic_state_derivative(P, ystar, u)
    assert np.max(np.abs(dY_free - dY)) > 1e-3 * np.max(np.abs(dY))


def test_plausible_mistakes_fail_the_difference_pins(setup):
    # each variant is one slip in writing the stacked system; every one must miss the
    # Richardson differences of the Newton solves by far more than the pins' tolerance
    p, P, u, ystar, solve = setup
    Jy, Ju = implicit.year_jacobians(P, ystar, u)
    N = ystar.size
    w = np.tile(p.vol, ystar.shape[0])
    w = w / np.linalg.norm(w)

    def stacked(A, rhs):
        return np.linalg.lstsq(np.vstack([A, w[None, :]]), np.vstack([rhs, np.zeros((1, rhs.shape[1]))]),
                               rcond=None)[0]

    fd = np.stack([richardson(lambda uu: solve(uu, ystar).ravel(), u, k) for k in range(u.size)], axis=1)
    good = stacked(np.eye(N) - Jy, Ju)
    assert np.max(np.abs(good - fd)) <= 1e-5 * np.max(np.abs(fd))
    mutants = {
        "transposed Jacobian": stacked(np.eye(N) - Jy.T, Ju),
        "sign of phi_y": stacked(np.eye(N) + Jy, Ju),
        "sign of phi_u": stacked(np.eye(N) - Jy, -Ju),
        "phi_y without the identity": stacked(-Jy, Ju),
    }
    for name, dY in mutants.items():
        assert np.max(np.abs(dY - fd)) > 1e-2 * np.max(np.abs(fd)), name
