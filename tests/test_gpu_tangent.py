"""The tangent year map on the GPU against the oracle's own tangent, and Newton with exact products."""
import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from oracle import newton as on
from tests._util import normwise_err, rel_err

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


@pytest.mark.parametrize("name,nsub", [("tiny_6x4x4", 1), ("tiny_6x4x4", 8), ("ndop_64x32x8", 1)])
@pytest.mark.parametrize("plan", ["resident", "persistent"])
def test_year_tangent_matches_oracle(m3d, name, nsub, plan):
    p = mi.make_problem(name)
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    v = mi.random_state(p, seed=5) - mi.random_state(p, seed=6)
    ctx = m3d.Context.from_problem(p, nsub=nsub)
    ctx.set_option(m3d.OPT_YEAR_PLAN, m3d.PLAN_RESIDENT if plan == "resident" else m3d.PLAN_PERSISTENT)
    phi = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    jv = torch.empty_like(phi)
    ctx.year_tangent(cuda(y), cuda(v), cuda(u), phi, jv)
    ctx.sync()
    want_phi, want_jv = oracle.year_tangent(P, y, v, u, nsub=nsub)
    assert rel_err(phi.cpu().numpy(), want_phi) < 1e-10
    assert np.abs(jv.cpu().numpy() - want_jv).max() / np.abs(want_jv).max() < 1e-10
    ctx.close()


def test_newton_with_tangent_products(m3d):
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y0 = mi.initial_state(p)
    ctx = m3d.Context.from_problem(p)
    y = cuda(y0)
    st, rep = ctx.newton_solve(y, cuda(u), tol=1e-8, jv=m3d.JV_TANGENT)
    assert st == m3d.M3D_OK and rep["tangent_maps"] > 0
    want, _ = on.newton_krylov(P, y0, u, tol=1e-8)
    assert np.abs(y.cpu().numpy() - want).max() / np.abs(want).max() < 1e-7
    ctx.close()


def test_year_tangent_matches_oracle_benchmark_grid(m3d):
    """The benchmark's 128 x 64 x 15 grid (52,749 cells), default plan and options: phi(y) and
    phi'(y) v element by element against the oracle's tangent year map (run on all host cores)."""
    import os
    p = mi.make_problem("ndop_128x64x15")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    v = mi.random_state(p, seed=5) - mi.random_state(p, seed=6)
    ctx = m3d.Context.from_problem(p)
    phi = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    jv = torch.empty_like(phi)
    ctx.year_tangent(cuda(y), cuda(v), cuda(u), phi, jv)
    ctx.sync()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        want_phi, want_jv = oracle.year_tangent(P, y, v, u)
    finally:
        oracle.set_threads(1)
    assert rel_err(phi.cpu().numpy(), want_phi) < 1e-10
    # phi'(y) v of a signed v changes sign across the grid: measured normwise (an element near
    # a sign change shows rounding of 1e-15 max|o| as a relative error of 1e-9)
    assert normwise_err(jv.cpu().numpy(), want_jv) < 1e-10
    ctx.close()


@pytest.mark.parametrize("name", ["tiny_6x4x4", "tiny_4x3x3", "ndop_64x32x8", "ndop_128x64x15"])
def test_linearised_tangent_matches_oracle(m3d, name):
    """phi'(y) v by the linearised sweep (the year map recording df/dN, then one sweep of the
    perturbation alone) against the oracle's tangent year map, and against the one-pass
    tangent on dual numbers."""
    import os
    p = mi.make_problem(name)
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    v = mi.random_state(p, seed=5) - mi.random_state(p, seed=6)
    ctx = m3d.Context.from_problem(p)
    phi = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    jv = torch.empty_like(phi)
    ctx.year_tangent(cuda(y), cuda(v), cuda(u), phi, jv)          # dual numbers (default)
    ctx.sync()
    jv_dual = jv.cpu().numpy()
    assert ctx.get_option(m3d.OPT_TANGENT_FORM) == m3d.TANGENT_DUAL
    ctx.set_option(m3d.OPT_TANGENT_FORM, m3d.TANGENT_LINEARISED)
    ctx.year_tangent(cuda(y), cuda(v), cuda(u), phi, jv)
    ctx.sync()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        want_phi, want_jv = oracle.year_tangent(P, y, v, u)
    finally:
        oracle.set_threads(1)
    assert rel_err(phi.cpu().numpy(), want_phi) < 1e-10
    assert normwise_err(jv.cpu().numpy(), want_jv) < 1e-10
    assert normwise_err(jv.cpu().numpy(), jv_dual) < 1e-10
    ctx.close()


def test_linearised_tangent_needs_one_internal_step(m3d):
    p = mi.make_problem("tiny_6x4x4")
    ctx = m3d.Context.from_problem(p, nsub=8)
    with pytest.raises(m3d.Metos3dError):
        ctx.set_option(m3d.OPT_TANGENT_FORM, m3d.TANGENT_LINEARISED)
    ctx.close()
