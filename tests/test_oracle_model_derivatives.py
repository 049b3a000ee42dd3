"""Pins of the oracle's tangents and reverses of the N, PO4-DOP-PHY and NPZD-DOP models.

The derivatives are written out by hand in the oracle (the paper's Section 6 names exact
derivatives by algorithmic differentiation as the alternative to finite differences); here
they are checked against central differences of the oracle's own forward model (which its
own pins fix), and the reverses against the tangents by the dot-product identity
<w, J v> = <J^T w, v>.  At the level of the year map the same checks run on a tiny grid.
"""
import math

import numpy as np
import pytest

import m3d_inputs as mi
import oracle

MODELS = [(oracle.MODEL_N, 1), (oracle.MODEL_NDOP, 2), (oracle.MODEL_PHY, 3), (oracle.MODEL_NPZD, 5)]


def column(L, seed):
    r = np.random.default_rng(seed)
    h = np.array([50.0 * 10 ** (k / 7) for k in range(L)])
    d = np.cumsum(h) - 0.5 * h
    return h, d, r


def params(model):
    return np.asarray(mi.default_params(model), dtype=np.float64)


@pytest.mark.parametrize("model,ntr", MODELS)
@pytest.mark.parametrize("L", [1, 2, 3, 8])
@pytest.mark.parametrize("nsub", [1, 3])
def test_bgc_tangent_matches_central_differences(model, ntr, L, nsub):
    h, d, r = column(L, 10 * L + ntr)
    u = params(model)
    y = 0.5 + r.random((ntr, L))
    dy = r.standard_normal((ntr, L))
    kw = dict(insol=300.0, model=model, nsub=nsub, dt=1.0 / 2880)
    q0, dq = oracle.bgc_tangent(y, dy, h, d, u, **kw)
    assert np.allclose(q0, oracle.bgc(y, h, d, u, **kw), rtol=0, atol=1e-16 * np.abs(q0).max() + 1e-300)
    eps = 1e-6
    fd = (oracle.bgc(y + eps * dy, h, d, u, **kw) - oracle.bgc(y - eps * dy, h, d, u, **kw)) / (2 * eps)
    # (a one-layer column of the N model keeps its whole production: q = 0 and so is dq)
    scale = max(np.abs(fd).max(), np.abs(dy).max() * 1e-9)
    # the increment is y^(nsub) - y^(0), so the differences carry rounding of eps(|y|) / eps each
    assert np.abs(dq - fd).max() <= 1e-7 * scale + 1e-9 * np.abs(y).max()


@pytest.mark.parametrize("model,ntr", MODELS)
@pytest.mark.parametrize("L", [1, 2, 3, 8])
@pytest.mark.parametrize("nsub", [1, 3])
def test_bgc_adjoint_is_the_transpose_of_the_tangent(model, ntr, L, nsub):
    h, d, r = column(L, 20 * L + ntr)
    u = params(model)
    y = 0.5 + r.random((ntr, L))
    v = r.standard_normal((ntr, L))
    w = r.standard_normal((ntr, L))
    kw = dict(insol=250.0, model=model, nsub=nsub)
    _, jv = oracle.bgc_tangent(y, v, h, d, u, **kw)
    ybar, ubar = oracle.bgc_adjoint(y, w, h, d, u, **kw)
    lhs, rhs = float(np.sum(w * jv)), float(np.sum(ybar * v))
    assert math.isclose(lhs, rhs, rel_tol=1e-12, abs_tol=1e-16 * np.abs(w).sum() * np.abs(jv).max())
    # the parameter part against central differences of <w, bgc(y; u)> in each parameter
    for k in range(u.size):
        hk = 1e-6 * max(abs(u[k]), 1e-3)
        up, um = u.copy(), u.copy()
        up[k] += hk
        um[k] -= hk
        fd = (np.sum(w * oracle.bgc(y, h, d, up, **kw)) - np.sum(w * oracle.bgc(y, h, d, um, **kw))) / (2 * hk)
        # the increment is y^(nsub) - y^(0): each evaluation carries rounding eps(|y|) per entry
        noise = 4e-16 * np.abs(y).max() * np.abs(w).sum() / hk
        assert abs(ubar[k] - fd) <= 1e-6 * abs(fd) + noise, (k, ubar[k], fd)


@pytest.fixture(scope="module")
def tiny():
    p = mi.make_problem("tiny_4x3x3")
    return p, oracle.Problem(p)


@pytest.mark.parametrize("model,ntr", MODELS)
def test_year_tangent_and_adjoint_of_every_model(tiny, model, ntr):
    """The year map's tangent against central differences, and its reverse against the
    tangent (dot product) and against central differences in the parameters."""
    p, P = tiny
    u = params(model)
    r = np.random.default_rng(ntr)
    y = mi.initial_state(p, ntr, mi.model_initial_values(model)) * (0.5 + r.random((ntr, p.n)))
    v = r.standard_normal((ntr, p.n))
    w = r.standard_normal((ntr, p.n))
    y1, jv = oracle.year_tangent(P, y, v, u, model=model)
    assert np.allclose(y1, oracle.year_map(P, y, u, model=model), rtol=1e-14, atol=0)
    # the NPZD-DOP year amplifies strongly: central differences converge as eps^2 (4e-6 at
    # 1e-6, 4e-8 at 1e-7) down to rounding near 1e-8
    eps = 1e-7 * np.linalg.norm(y) / np.linalg.norm(v)
    fd = (oracle.year_map(P, y + eps * v, u, model=model) - oracle.year_map(P, y - eps * v, u, model=model)) / (2 * eps)
    assert np.abs(jv - fd).max() <= 1e-6 * np.abs(fd).max()
    ybar, ubar = oracle.year_adjoint(P, y, u, w, model=model)
    assert math.isclose(float(np.sum(w * jv)), float(np.sum(ybar * v)), rel_tol=1e-11)
    def central(k, hk):
        up, um = u.copy(), u.copy()
        up[k] += hk
        um[k] -= hk
        return (np.sum(w * oracle.year_map(P, y, up, model=model)) -
                np.sum(w * oracle.year_map(P, y, um, model=model))) / (2 * hk)

    for k in range(u.size):
        # Richardson's extrapolation of central differences at h and h/2 cancels their h^2 term
        hk = 1e-4 * abs(u[k])
        fdk = (4.0 * central(k, hk / 2) - central(k, hk)) / 3.0
        assert abs(ubar[k] - fdk) <= 1e-6 * max(abs(fdk), 1e-8 * np.abs(w).sum()), (k, ubar[k], fdk)
