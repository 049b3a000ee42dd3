"""Pins of the oracle's adjoint year map: the dot-product test against the oracle's tangent
(<w, phi_y v> = <phi_y^T w, v>) and central finite differences for the parameter gradient."""
import numpy as np
import pytest

import m3d_inputs as mi
import oracle


@pytest.fixture(scope="module")
def tiny():
    p = mi.make_problem("tiny_6x4x4")
    return p, oracle.Problem(p)


def _col(nl):
    h = np.array([50.0, 70.0, 100.0, 140.0, 190.0, 240.0, 290.0, 340.0])[:nl]
    return h, np.cumsum(h) - 0.5 * h


@pytest.mark.parametrize("nl", [1, 2, 3, 8])
@pytest.mark.parametrize("nsub", [1, 8])
def test_bgc_adjoint_dot_product_and_parameter_gradient(nl, nsub):
    r = np.random.default_rng(3 * nl + nsub)
    h, d = _col(nl)
    u = mi.default_params_ndop() * r.uniform(0.7, 1.3, 7)
    y = r.uniform(0.1, 3.0, (2, nl))
    insol = r.uniform(50, 500)
    for _ in range(3):
        v = r.standard_normal((2, nl))
        wbar = r.standard_normal((2, nl))
        _, jv = oracle.bgc_tangent(y, v, h, d, u, insol=insol, nsub=nsub)
        ybar, ubar = oracle.bgc_adjoint(y, wbar, h, d, u, insol=insol, nsub=nsub)
        lhs, rhs = float(np.sum(wbar * jv)), float(np.sum(ybar * v))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(wbar).sum() * np.abs(jv).max())
        for k in range(7):                                   # d <wbar, bgc(u)> / du_k
            e = 1e-6 * u[k]
            up, um = u.copy(), u.copy()
            up[k] += e
            um[k] -= e
            fd = float(np.sum(wbar * (oracle.bgc(y, h, d, up, insol=insol, nsub=nsub) -
                                      oracle.bgc(y, h, d, um, insol=insol, nsub=nsub)))) / (2 * e)
            # bgc returns y^(nsub) - y^(0), rounded at eps |y|: that noise, divided by 2e, bounds the FD error
            noise = 8 * nsub * np.finfo(float).eps * np.abs(wbar).sum() * np.abs(y).max() / e
            assert abs(ubar[k] - fd) <= 1e-6 * abs(fd) + noise, (k, ubar[k], fd)


def test_year_adjoint_dot_product(tiny):
    p, P = tiny
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    v = mi.random_state(p, seed=5) - mi.random_state(p, seed=6)
    wbar = mi.random_state(p, seed=8) - 1.0
    _, jv = oracle.year_tangent(P, y, v, u)
    ybar0, _ = oracle.year_adjoint(P, y, u, wbar)
    lhs, rhs = float(np.sum(wbar * jv)), float(np.sum(ybar0 * v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_year_adjoint_parameter_gradient_matches_central_differences(tiny):
    p, P = tiny
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    wbar = mi.random_state(p, seed=8) - 1.0
    _, ubar = oracle.year_adjoint(P, y, u, wbar)
    for k in range(7):
        e = 1e-6 * u[k]
        up, um = u.copy(), u.copy()
        up[k] += e
        um[k] -= e
        fd = float(np.sum(wbar * (oracle.year_map(P, y, up) - oracle.year_map(P, y, um)))) / (2 * e)
        assert abs(ubar[k] - fd) <= 1e-6 * abs(fd) + 1e-10, (k, ubar[k], fd)


def test_adjoint_of_pure_transport_is_the_transpose(tiny):
    p, P = tiny
    y = mi.random_state(p, ntracer=1)
    v = mi.random_state(p, ntracer=1, seed=2)
    w = mi.random_state(p, ntracer=1, seed=4)
    phi_v = oracle.year_map(P, v, np.zeros(0), model=oracle.MODEL_NONE)
    wbar0, _ = oracle.year_adjoint(P, y, np.zeros(0), w, model=oracle.MODEL_NONE)
    assert abs(float(np.sum(w * phi_v)) - float(np.sum(wbar0 * v))) <= 1e-13 * abs(float(np.sum(w * phi_v)))
