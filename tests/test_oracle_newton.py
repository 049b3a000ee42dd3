"""Pins of the oracle's spin-up and Newton-Krylov solve (Sections 4, 6, 7).

Newton's method and the spin-up (plain fixed-point iteration of the year map) are different
algorithms for the same periodic solution; for a fixed total mass it is unique.
"""
import math

import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from oracle import newton as on


@pytest.fixture(scope="module")
def tiny():
    p = mi.make_problem("tiny_6x4x4")
    return p, oracle.Problem(p)


@pytest.fixture(scope="module")
def newton_solution(tiny):
    p, P = tiny
    y0 = mi.initial_state(p)
    y, rep = on.newton_krylov(P, y0, mi.default_params_ndop(), tol=1e-8)
    return y0, y, rep


def test_gmres_mgs_solves_a_small_system():
    r = np.random.default_rng(0)
    A = np.eye(30) + 0.3 * r.standard_normal((30, 30)) / math.sqrt(30)
    b = r.standard_normal(30)
    for restart in (30, 7):                  # full and restarted
        x, it, res = on.gmres_mgs(lambda v: A @ v, b, 1e-12, restart, 500)
        assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)


def test_newton_converges_and_keeps_mass(tiny, newton_solution):
    p, P = tiny
    y0, y, rep = newton_solution
    assert rep["converged"] and rep["residuals"][-1] < 1e-8
    assert len(rep["residuals"]) <= 12
    # the residual really is ||phi(y) - y|| at the returned state
    py = oracle.year_map(P, y, mi.default_params_ndop())
    assert np.linalg.norm((py - y).ravel()) < 1e-8
    m0 = math.fsum((p.vol * y0).ravel())
    assert abs(math.fsum((p.vol * y).ravel()) / m0 - 1) < 1e-13


@pytest.mark.slow
def test_newton_agrees_with_long_spinup(tiny, newton_solution):
    """The paper's comparison: spin-up (fixed-point iteration) and Newton reach the same periodic state."""
    p, P = tiny
    y0, y, _ = newton_solution
    ys, hist = on.spinup(P, y0, mi.default_params_ndop(), 1500)
    assert hist[-1] < 1e-11
    big = [h for h in hist if h > 1e-10]                # above the rounding floor the decay is monotone
    assert hist[0] > 1.0 and all(b < a * 1.0001 for a, b in zip(big[50:], big[51:]))
    assert np.abs(ys - y).max() / np.abs(y).max() < 1e-7


def test_tangent_product_option_matches_fd(tiny):
    """With an exact phi'(y) v (here: central differences of the oracle), Newton converges too."""
    p, P = tiny
    u = mi.default_params_ndop()

    def jv(y, py, v):
        h = 1e-6 * np.linalg.norm(y) / np.linalg.norm(v)
        return (oracle.year_map(P, y + h * v, u) - oracle.year_map(P, y - h * v, u)) / (2 * h)

    y, rep = on.newton_krylov(P, mi.initial_state(p), u, tol=1e-8, jv=jv)
    assert rep["converged"]
