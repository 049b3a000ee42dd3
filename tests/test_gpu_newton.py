"""Spin-up and Newton-Krylov on the GPU (Sections 4, 6, 7) against the oracle."""
import math

import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from oracle import newton as on
from tests._util import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_spinup_matches_oracle(m3d):
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    ctx = m3d.Context.from_problem(p)
    y = cuda(mi.initial_state(p))
    res = ctx.spinup(y, cuda(u), 20)
    ys, hist = on.spinup(P, mi.initial_state(p), u, 20)
    assert rel_err(y.cpu().numpy(), ys) < 1e-10
    assert np.allclose(res, hist, rtol=1e-8, atol=1e-12)
    ctx.close()


def test_newton_matches_oracle_newton_tiny(m3d):
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y0 = mi.initial_state(p)
    ctx = m3d.Context.from_problem(p)
    y = cuda(y0)
    st, rep = ctx.newton_solve(y, cuda(u), tol=1e-8)
    assert st == m3d.M3D_OK and rep["converged"] and rep["residual"] < 1e-8
    want, orep = on.newton_krylov(P, y0, u, tol=1e-8)
    got = y.cpu().numpy()
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-7       # the same periodic solution
    m0 = math.fsum((p.vol * y0).ravel())
    assert abs(math.fsum((p.vol * got).ravel()) / m0 - 1) < 1e-12    # mass kept
    # the oracle's own year map confirms the fixed point
    assert np.linalg.norm((oracle.year_map(P, got, u) - got).ravel()) < 2e-8
    ctx.close()


def test_newton_64x32x8_is_a_fixed_point_of_the_oracle(m3d):
    p = mi.make_problem("ndop_64x32x8")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y0 = mi.initial_state(p)
    ctx = m3d.Context.from_problem(p)
    y = cuda(y0)
    st, rep = ctx.newton_solve(y, cuda(u), tol=1e-8)
    assert st == m3d.M3D_OK, rep
    got = y.cpu().numpy()
    assert np.linalg.norm((oracle.year_map(P, got, u) - got).ravel()) < 5e-8
    assert got.min() > 0.0
    ctx.close()


def test_newton_reports_not_converged(m3d):
    p = mi.make_problem("tiny_4x3x3")
    ctx = m3d.Context.from_problem(p)
    y = cuda(mi.initial_state(p))
    st, rep = ctx.newton_solve(y, cuda(mi.default_params_ndop()), max_newton=1, tol=1e-12)
    assert st == m3d.M3D_NOT_CONVERGED and not rep["converged"] and rep["newton_steps"] == 1
    ctx.close()
