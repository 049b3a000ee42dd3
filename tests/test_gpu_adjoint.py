"""The adjoint year map on the GPU: against the oracle's adjoint, the GPU tangent (dot-product
test), central finite differences of the parameter gradient, and through torch.autograd."""
import numpy as np
import pytest

import m3d_inputs as mi
import oracle

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


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name", ["tiny_6x4x4", "ndop_64x32x8"])
@pytest.mark.parametrize("form", ["tridiagonal", "dense"])
def test_adjoint_matches_oracle(m3d, name, form):
    p = mi.make_problem(name)
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y0 = mi.random_state(p)
    wbar = mi.random_state(p, seed=8) - 1.0
    ctx = m3d.Context.from_problem(p)
    if form == "dense":
        ctx.set_option(m3d.OPT_IMPLICIT_FORM, m3d.IMPLICIT_DENSE)
    ybar0 = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    ubar = ctx.year_adjoint(cuda(y0), cuda(u), cuda(wbar), ybar0)
    want_y, want_u = oracle.year_adjoint(P, y0, u, wbar)
    assert rel(ybar0.cpu().numpy(), want_y) < 1e-10
    assert np.abs(ubar - want_u).max() <= 1e-9 * np.abs(want_u).max()
    ctx.close()


def test_adjoint_dot_product_with_gpu_tangent(m3d):
    p = mi.make_problem("ndop_64x32x8")
    u = cuda(mi.default_params_ndop())
    y0 = cuda(mi.random_state(p))
    v = cuda(mi.random_state(p, seed=5) - mi.random_state(p, seed=6))
    w = cuda(mi.random_state(p, seed=8) - 1.0)
    ctx = m3d.Context.from_problem(p)
    phi = torch.empty_like(y0)
    jv = torch.empty_like(y0)
    ctx.year_tangent(y0, v, u, phi, jv)
    wbar0 = torch.empty_like(y0)
    ctx.year_adjoint(y0, u, w, wbar0)
    ctx.sync()
    lhs = float(torch.sum(w * jv))
    rhs = float(torch.sum(wbar0 * v))
    assert abs(lhs - rhs) <= 1e-12 * float(torch.sum(torch.abs(w) * torch.abs(jv)))
    ctx.close()


@pytest.mark.parametrize("ckpt", [240, 100, 2880])
def test_checkpoint_interval_does_not_change_the_result(m3d, ckpt):
    p = mi.make_problem("tiny_6x4x4")
    u = cuda(mi.default_params_ndop())
    y0 = cuda(mi.random_state(p))
    w = cuda(mi.random_state(p, seed=8) - 1.0)
    ctx = m3d.Context.from_problem(p)
    ref = torch.empty_like(y0)
    ub_ref = ctx.year_adjoint(y0, u, w, ref, 240)
    got = torch.empty_like(y0)
    ub = ctx.year_adjoint(y0, u, w, got, ckpt)
    assert torch.equal(ref, got)
    # the parameter gradient is summed segment by segment: equal up to the grouping of the sum
    assert np.allclose(ub, ub_ref, rtol=1e-13, atol=0)
    ctx.close()


def test_misfit_gradient_matches_central_differences(m3d):
    """The parameter optimisation's gradient: J(u) = 1/2 |M (phi(y0; u) - obs)|^2 on a random 10 %
    of the cells, observations from perturbed parameters plus 5 % noise."""
    p = mi.make_problem("ndop_64x32x8")
    r = mi.rng(1410, "observations")
    u0 = mi.default_params_ndop()
    y0 = cuda(mi.random_state(p))
    ctx = m3d.Context.from_problem(p)
    mask = torch.from_numpy((r.random((2, p.n)) < 0.1).astype(np.float64)).cuda()
    u_true = cuda(u0 * r.uniform(0.8, 1.2, 7))
    obs = torch.empty_like(y0)
    ctx.year_map(y0, obs, u_true)
    obs = obs * cuda(1.0 + 0.05 * r.standard_normal((2, p.n)))
    u = cuda(u0)

    def J(uu):
        y1 = torch.empty_like(y0)
        ctx.year_map(y0, y1, uu)
        return 0.5 * float(torch.sum((mask * (y1 - obs)) ** 2))

    y1 = torch.empty_like(y0)
    ctx.year_map(y0, y1, u)
    ybar1 = mask * mask * (y1 - obs)
    ybar0 = torch.empty_like(y0)
    grad = ctx.year_adjoint(y0, u, ybar1, ybar0)
    for k in range(7):
        e = 1e-6 * u0[k]
        up, um = u0.copy(), u0.copy()
        up[k] += e
        um[k] -= e
        fd = (J(cuda(up)) - J(cuda(um))) / (2 * e)
        assert abs(grad[k] - fd) <= 1e-5 * abs(fd) + 1e-9 * abs(J(u)), (k, grad[k], fd)
    ctx.close()


def test_autograd_function(m3d):
    p = mi.make_problem("tiny_6x4x4")
    ctx = m3d.Context.from_problem(p)
    y0 = cuda(mi.random_state(p)).requires_grad_(True)
    u = cuda(mi.default_params_ndop()).requires_grad_(True)
    w = cuda(mi.random_state(p, seed=8) - 1.0)
    y1 = m3d.year_map_autograd(y0, u, ctx)
    loss = torch.sum(w * y1)
    loss.backward()
    ybar0 = torch.empty_like(w)
    ubar = ctx.year_adjoint(y0.detach(), u.detach(), w, ybar0)
    assert torch.equal(y0.grad, ybar0)
    assert np.array_equal(u.grad.cpu().numpy(), ubar)
    ctx.close()


@pytest.mark.slow
def test_adjoint_matches_oracle_full_grid(m3d):
    # the benchmark's 128 x 64 x 15 grid, seeded state and cotangent, checkpoint every 240 steps
    import os
    oracle.set_threads(min(16, os.cpu_count() or 1))
    p = mi.make_problem("ndop_128x64x15")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y0 = mi.random_state(p, seed=21)
    wbar = mi.random_state(p, seed=22) - 1.0
    ctx = m3d.Context.from_problem(p)
    ybar0 = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    ubar = ctx.year_adjoint(cuda(y0), cuda(u), cuda(wbar), ybar0, 240)
    want_y, want_u = oracle.year_adjoint(P, y0, u, wbar)
    oracle.set_threads(1)
    assert rel(ybar0.cpu().numpy(), want_y) < 1e-10
    assert np.abs(ubar - want_u).max() <= 1e-9 * np.abs(want_u).max()
    ctx.close()


@pytest.mark.slow
def test_misfit_gradient_at_the_periodic_solution_full_grid(m3d):
    """The parameter-optimisation gradient on the benchmark grid: observations are the periodic
    solution at seeded perturbed parameters plus 5 % Gaussian noise on a random 10 % of the
    wet cells; J(u) = 1/2 |M (phi(y*; u) - obs)|^2 from the periodic solution y* of the
    default parameters (held fixed).  The adjoint's gradient (checkpoint every 240 steps) must
    match central differences with h = 1e-6 relative."""
    p = mi.make_problem("ndop_128x64x15")
    r = mi.rng(1410, "observations")
    u0 = mi.default_params_ndop()
    u_true = u0 * r.uniform(0.9, 1.1, 7)
    ctx = m3d.Context.from_problem(p)
    periodic = {}
    for name, uu in (("true", u_true), ("default", u0)):
        y = cuda(mi.initial_state(p))
        st, rep = ctx.newton_solve(y, cuda(uu), tol=1e-8)
        assert rep["converged"], name
        periodic[name] = y
    mask = cuda((r.random((2, p.n)) < 0.1).astype(np.float64))
    obs = periodic["true"] * cuda(1.0 + 0.05 * r.standard_normal((2, p.n)))
    ystar = periodic["default"]

    def J(uu):
        y1 = torch.empty_like(ystar)
        ctx.year_map(ystar, y1, cuda(uu))
        return 0.5 * float(torch.sum((mask * (y1 - obs)) ** 2))

    y1 = torch.empty_like(ystar)
    ctx.year_map(ystar, y1, cuda(u0))
    ybar1 = mask * mask * (y1 - obs)
    grad = ctx.year_adjoint(ystar, cuda(u0), ybar1, torch.empty_like(ystar), 240)
    J0 = J(u0)
    for k in range(7):
        e = 1e-6 * u0[k]
        up, um = u0.copy(), u0.copy()
        up[k] += e
        um[k] -= e
        fd = (J(up) - J(um)) / (2 * e)
        assert abs(grad[k] - fd) <= 1e-5 * abs(fd) + 1e-9 * J0, (k, grad[k], fd)
    ctx.close()


@pytest.mark.parametrize("name", ["ndop_64x32x8", "ndop_128x64x15"])
def test_streaming_adjoint_matches_oracle(m3d, name):
    # the sweep that reads its operators from HBM (what grids too large for the resident
    # kernel use), forced on grids where the resident sweep also runs
    import os
    oracle.set_threads(min(16, os.cpu_count() or 1))
    p = mi.make_problem(name)
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    y0 = mi.random_state(p, seed=31)
    wbar = mi.random_state(p, seed=32) - 1.0
    ctx = m3d.Context.from_problem(p)
    assert ctx.get_option(m3d.OPT_ADJOINT_PLAN) == m3d.PLAN_RESIDENT
    ctx.set_option(m3d.OPT_ADJOINT_PLAN, m3d.PLAN_PERSISTENT)
    assert ctx.get_option(m3d.OPT_ADJOINT_PLAN) == m3d.PLAN_PERSISTENT
    ybar0 = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    ubar = ctx.year_adjoint(cuda(y0), cuda(u), cuda(wbar), ybar0, 240)
    want_y, want_u = oracle.year_adjoint(P, y0, u, wbar)
    oracle.set_threads(1)
    assert rel(ybar0.cpu().numpy(), want_y) < 1e-10
    assert np.abs(ubar - want_u).max() <= 1e-9 * np.abs(want_u).max()
    # and the resident sweep agrees with it to rounding (dense against tridiagonal implicit form)
    ctx.set_option(m3d.OPT_ADJOINT_PLAN, m3d.PLAN_RESIDENT)
    ybar_r = torch.empty_like(ybar0)
    ubar_r = ctx.year_adjoint(cuda(y0), cuda(u), cuda(wbar), ybar_r, 240)
    assert rel(ybar0.cpu().numpy(), ybar_r.cpu().numpy()) < 1e-11
    assert np.abs(ubar - ubar_r).max() <= 1e-10 * np.abs(ubar_r).max()
    ctx.close()


def test_reverse_sweep_step_operators_bit_identical_and_abort(m3d):
    """The reverse sweep streaming per-step transposed operators gives the bits of the sweep
    that interpolates every entry in the kernel (both checkpoint intervals); a withheld tile
    makes it time out (its bulk copies in flight land first) and the context works on."""
    p = mi.make_problem("ndop_64x32x8")
    u = cuda(mi.default_params_ndop())
    y0 = cuda(mi.random_state(p))
    wbar = cuda(mi.random_state(p, seed=8) - 1.0)
    ctx = m3d.Context.from_problem(p)
    assert ctx.get_option(m3d.OPT_STEP_OPERATORS) == 1
    got = {}
    for stepop in (1, 0):
        ctx.set_option(m3d.OPT_STEP_OPERATORS, stepop)
        for ckpt in (240, p.nstep):
            yb = torch.empty_like(y0)
            ub = ctx.year_adjoint(y0, u, wbar, yb, ckpt)
            got[(stepop, ckpt)] = (yb.cpu().numpy(), ub)
    for ckpt in (240, p.nstep):
        assert np.array_equal(got[(1, ckpt)][0], got[(0, ckpt)][0]), ckpt
        assert np.array_equal(got[(1, ckpt)][1], got[(0, ckpt)][1]), ckpt
    ctx.set_option(m3d.OPT_STEP_OPERATORS, 1)
    ctx.set_option(m3d.OPT_WAIT_TIMEOUT_NS, 50_000_000)      # 50 ms
    ctx.set_option(m3d.OPT_TEST_WITHHOLD_TILE, 0)
    with pytest.raises(m3d.Metos3dError) as e:
        ctx.year_adjoint(y0, u, wbar, torch.empty_like(y0), 240)
    assert e.value.status == m3d.M3D_ERR_TIMEOUT
    ctx.set_option(m3d.OPT_TEST_WITHHOLD_TILE, -1)
    ctx.set_option(m3d.OPT_WAIT_TIMEOUT_NS, 2_000_000_000)
    yb = torch.empty_like(y0)
    ub = ctx.year_adjoint(y0, u, wbar, yb, 240)
    assert np.array_equal(yb.cpu().numpy(), got[(1, 240)][0]) and np.array_equal(ub, got[(1, 240)][1])
    ctx.close()
