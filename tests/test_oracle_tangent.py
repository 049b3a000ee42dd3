"""Pins of the oracle's tangent-linear year map (Section 6: exact Jacobian-vector products)."""
import math

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
def test_bgc_tangent_matches_central_differences(nl, nsub):
    r = np.random.default_rng(11 * nl + nsub)
    h, d = _col(nl)
    for _ in range(5):
        u = mi.default_params_ndop() * r.uniform(0.5, 1.5, 7)
        y = r.uniform(0.1, 3.0, (2, nl))
        dy = r.standard_normal((2, nl))
        insol = r.uniform(50, 500)
        yb, dyb = oracle.bgc_tangent(y, dy, h, d, u, insol=insol, nsub=nsub)
        assert np.allclose(yb, oracle.bgc(y, h, d, u, insol=insol, nsub=nsub), rtol=0, atol=1e-15)
        eps = 1e-5
        fd = (oracle.bgc(y + eps * dy, h, d, u, insol=insol, nsub=nsub) -
              oracle.bgc(y - eps * dy, h, d, u, insol=insol, nsub=nsub)) / (2 * eps)
        assert np.abs(dyb - fd).max() <= 1e-7 * max(np.abs(dyb).max(), 1e-12) + 1e-12


def test_year_tangent_matches_central_differences(tiny):
    p, P = tiny
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    v = mi.random_state(p, seed=5) - mi.random_state(p, seed=6)
    y1, jv = oracle.year_tangent(P, y, v, u)
    assert np.array_equal(y1, oracle.year_map(P, y, u))
    hh = 1e-4
    fd = (oracle.year_map(P, y + hh * v, u) - oracle.year_map(P, y - hh * v, u)) / (2 * hh)
    assert np.abs(jv - fd).max() / np.abs(jv).max() < 1e-7


def test_tangent_of_pure_transport_is_the_map_itself(tiny):
    p, P = tiny
    y = mi.random_state(p, ntracer=3)
    v = mi.random_state(p, ntracer=3, seed=9)
    _, jv = oracle.year_tangent(P, y, v, np.zeros(0), model=oracle.MODEL_NONE)
    phi_v = oracle.year_map(P, v, np.zeros(0), model=oracle.MODEL_NONE)
    assert np.abs(jv - phi_v).max() / np.abs(phi_v).max() < 1e-14


def test_tangent_conserves_mass_and_is_linear(tiny):
    p, P = tiny
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    v = mi.random_state(p, seed=3) - 0.9 * mi.random_state(p, seed=4)
    w = mi.random_state(p, seed=7)
    _, jv = oracle.year_tangent(P, y, v, u)
    _, jw = oracle.year_tangent(P, y, w, u)
    _, jvw = oracle.year_tangent(P, y, 2.0 * v - 3.0 * w, u)
    assert np.abs(jvw - (2.0 * jv - 3.0 * jw)).max() / np.abs(jvw).max() < 1e-13
    mv = math.fsum((p.vol * v).ravel())
    scale = math.fsum((p.vol * np.abs(v)).ravel())
    assert abs(math.fsum((p.vol * jv).ravel()) - mv) / scale < 1e-12
