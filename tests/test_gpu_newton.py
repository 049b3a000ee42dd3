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


def test_newton_backtracking_matches_oracle_step_by_step(m3d):
    """A far start (N x 10, alpha x 1.5) on which the line search backtracks with both the
    quadratic and the cubic model.  With tangent products on both sides the GPU solve
    follows the oracle's step by step: the same GMRES iteration counts, forcing terms, slopes,
    step lengths tried and accepted, and the same periodic state."""
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = mi.default_params_ndop() * np.array((1.0, 1.5, 1.0, 1.0, 1.0, 1.0, 1.0))
    y0 = mi.initial_state(p) * np.array((10.0, 1.0))[:, None]
    ctx = m3d.Context.from_problem(p)
    y = cuda(y0)
    st, rep = ctx.newton_solve(y, cuda(u), tol=1e-8, jv=m3d.JV_TANGENT)
    assert st == m3d.M3D_OK and rep["converged"], rep

    def tan(yy, py, v):
        return oracle.year_tangent(P, yy, v, u)[1]

    want, orep = on.newton_krylov(P, y0, u, tol=1e-8, jv=tan)
    assert rep["newton_steps"] == len(orep["krylov"])
    assert rep["krylov"] == orep["krylov"]
    assert [len(t) for t in rep["trials"]] == [len(t) for t in orep["trials"]]
    # Values: the two solves differ by rounding, and each backtrack fits its model to
    # differences of f values that cancel, so the differences grow along the backtracking path
    # (2e-7 in eta over the first steps, 1e-2 in the step length by the seventh): compared at
    # 1e-5 over the first five steps; after them the iteration counts and step counts above,
    # and the solution below, are the comparison.
    for k in range(5):
        for key in ("etas", "slopes", "lambdas"):
            assert np.isclose(rep[key][k], orep[key][k], rtol=1e-5, atol=0), (key, k, rep[key][k], orep[key][k])
        assert np.allclose(rep["trials"][k], orep["trials"][k], rtol=1e-5, atol=0), k
    assert min(rep["lambdas"]) < 0.5 and max(len(t) for t in rep["trials"]) >= 3
    got = y.cpu().numpy()
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-7
    ctx.close()


def npzd_far_start(p, scale_p):
    """NPZD-DOP's constant start with the phytoplankton scaled: full Newton steps from it leave
    the model's domain (negative zooplankton under quadratic mortality overflows within the year)."""
    return mi.initial_state(p, 5, mi.model_initial_values(mi.MODEL_NPZD)) * \
        np.array((1.0, scale_p, 1.0, 1.0, 1.0))[:, None]


def oracle_npzd_newton(P, y0, u, steps, krylov):
    def tan(yy, py, v):
        return oracle.year_tangent(P, yy, v, u, model=mi.MODEL_NPZD)[1]
    return on.newton_krylov(P, y0, u, tol=1e-8, max_newton=steps, restart=krylov, max_krylov=krylov,
                            model=mi.MODEL_NPZD, jv=tan, record_steps=True)


def test_newton_line_search_through_trials_that_overflow(m3d):
    """NPZD-DOP (phytoplankton x 10, three Krylov iterations per step, tangent products): the
    full step of the first Newton step and its tenth both overflow the year map, the third
    trial decreases |F|; the third step's full step overflows again.  The GPU solve takes the
    oracle's trials (a non-finite trial is cut to a tenth and gives no model), the same
    residuals, and ends on a finite state."""
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = np.asarray(mi.default_params(mi.MODEL_NPZD), dtype=np.float64)
    y0 = npzd_far_start(p, 10.0)
    want, orep = oracle_npzd_newton(P, y0, u, 4, 3)
    # the oracle's own trials at lambda = 1 and 0.1 of the first step overflow
    s0 = orep["steps"][0].reshape(y0.shape)
    for lam in (1.0, 0.1):
        assert not np.isfinite(oracle.year_map(P, y0 + lam * s0, u, model=mi.MODEL_NPZD)).all()
    assert orep["trials"][0] == [1.0, 0.1, 0.010000000000000002] and len(orep["trials"][2]) == 2
    ctx = m3d.Context.from_problem(p, model=mi.MODEL_NPZD, ntracer=5, nparam=len(u))
    y = cuda(y0)
    st, rep = ctx.newton_solve(y, cuda(u), tol=1e-8, max_newton=4, restart=3, max_krylov=3, jv=m3d.JV_TANGENT)
    assert st == m3d.M3D_NOT_CONVERGED and not rep["line_search_failed"]
    assert rep["krylov"] == orep["krylov"]
    assert [len(t) for t in rep["trials"]] == [len(t) for t in orep["trials"]]
    for k in range(4):
        assert np.allclose(rep["trials"][k], orep["trials"][k], rtol=1e-6, atol=0), (k, rep["trials"], orep["trials"])
    assert np.allclose(rep["residuals"], orep["residuals"], rtol=1e-5, atol=0), (rep["residuals"], orep["residuals"])
    got = y.cpu().numpy()
    assert np.isfinite(got).all() and np.abs(got - want).max() / np.abs(want).max() < 1e-5
    ctx.close()


def test_newton_fd_backtracks_and_converges(m3d):
    """The same far start with finite-difference products: the line search backtracks and the
    solve reaches the oracle's periodic state."""
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = mi.default_params_ndop() * np.array((1.0, 1.5, 1.0, 1.0, 1.0, 1.0, 1.0))
    y0 = mi.initial_state(p) * np.array((10.0, 1.0))[:, None]
    ctx = m3d.Context.from_problem(p)
    y = cuda(y0)
    st, rep = ctx.newton_solve(y, cuda(u), tol=1e-8)
    assert st == m3d.M3D_OK and rep["converged"], rep
    assert min(rep["lambdas"]) < 1.0
    got = y.cpu().numpy()
    assert np.linalg.norm((oracle.year_map(P, got, u) - got).ravel()) < 2e-8
    ctx.close()
