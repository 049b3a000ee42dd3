"""The 1-degree grid: 360 x 180 x 23 (700,000 wet cells in 42,120 columns, ~9.8 M explicit entries).

At this size the oracle finishes a few steps in seconds, not a year, so the checks are
element-wise parity over a few steps (single context and the 16-member NPZD-DOP ensemble),
and, over a whole year, properties that hold at any size: each member's mass is conserved
and the state stays finite and positive.
"""
import os

import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from tests._util import rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

STEP_TOL = 1e-12
NAME = "npzd_360x180x23"


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    oracle.set_threads(min(16, os.cpu_count() or 1))
    yield m
    oracle.set_threads(1)


@pytest.fixture(scope="module")
def grid():
    p = mi.make_problem(NAME)
    assert p.n == 700000 and p.ncol == 42120 and p.lmax == 23
    return p, oracle.Problem(p)


def test_single_context_steps_match_oracle(m3d, grid):
    p, P = grid
    ctx = m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    y0 = mi.random_state(p, 2, seed=91)
    u = mi.default_params_ndop()
    yd = torch.from_numpy(y0).cuda()
    ud = torch.from_numpy(u).cuda()
    a, b = yd.clone(), torch.empty_like(yd)
    j0, nsteps = 1195, 4                                   # across the May/June boundary
    for s in range(nsteps):
        ctx.step(j0 + s, a, b, ud)
        a, b = b, a
    want = oracle.steps(P, j0, nsteps, y0, u)
    assert rel_err(a.cpu().numpy(), want) <= STEP_TOL
    ctx.close()


def test_single_context_year_conserves_mass(m3d, grid):
    p, _ = grid
    ctx = m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    y0 = torch.from_numpy(mi.initial_state(p)).cuda()
    u = torch.from_numpy(mi.default_params_ndop()).cuda()
    y1 = ctx.year_map(y0, torch.empty_like(y0), u)
    m0, m1 = ctx.mass(y0), ctx.mass(y1)
    assert abs(m1 - m0) <= 1e-12 * m0
    y1h = y1.cpu().numpy()
    assert np.all(np.isfinite(y1h)) and y1h.min() > 0.0
    ctx.close()


def test_tangent_year_matches_central_differences(m3d, grid):
    # the tangent's tiles hold four components, which fit in shared memory because the tiles
    # of a PO4-DOP context are capped at the cells that allow it; phi'(y) v against
    # (phi(y + h v) - phi(y - h v)) / 2h, and the tangent's phi against the year map
    p, _ = grid
    ctx = m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    y0 = torch.from_numpy(mi.random_state(p, 2, seed=77)).cuda()
    v = torch.from_numpy(mi.random_state(p, 2, seed=78) - 0.5).cuda()
    u = torch.from_numpy(mi.default_params_ndop()).cuda()
    phi, jv = torch.empty_like(y0), torch.empty_like(y0)
    ctx.year_tangent(y0, v, u, phi, jv)
    y1 = torch.empty_like(y0)
    ctx.year_map(y0, y1, u)
    h = 1e-6 * float(torch.linalg.norm(y0)) / float(torch.linalg.norm(v))
    yp, ym = torch.empty_like(y0), torch.empty_like(y0)
    ctx.year_map(y0 + h * v, yp, u)
    ctx.year_map(y0 - h * v, ym, u)
    fd = ((yp - ym) / (2 * h)).cpu().numpy()
    # the year map applies the implicit part in Thomas form, the tangent's four-component
    # tile the dense blocks: equal up to rounding
    assert rel_err(phi.cpu().numpy(), y1.cpu().numpy()) <= 1e-11
    assert np.max(np.abs(jv.cpu().numpy() - fd)) <= 1e-6 * np.max(np.abs(fd))
    ctx.close()


def test_npzd_ensemble_steps_match_oracle(m3d, grid):
    p, P = grid
    members = mi.make_ensemble(((mi.MODEL_NPZD, 16),), seed=5)
    ens = m3d.Ensemble.from_problem(p, members)
    assert ens.width == 80 and ens.ngroup == 3
    ys = [mi.random_state(p, 5, seed=200 + i, scale=(4.4, 0.07, 0.07, 0.07, 0.05)) for i in range(16)]
    Y0 = torch.from_numpy(np.vstack(ys)).cuda()
    j0, nsteps = 2878, 3                                   # across the year's end
    Y1 = ens.steps(j0, nsteps, Y0, torch.empty_like(Y0)).cpu().numpy()
    want = oracle.ensemble_steps(P, j0, nsteps, ys, members)
    for m in range(16):
        assert rel_err(Y1[5 * m:5 * m + 5], want[m]) <= STEP_TOL, m
    ens.close()


def test_npzd_ensemble_year_conserves_each_member(m3d, grid):
    p, _ = grid
    members = mi.make_ensemble(((mi.MODEL_NPZD, 16),), seed=6)
    ens = m3d.Ensemble.from_problem(p, members)
    ys = [mi.initial_state(p, 5, mi.model_initial_values(mi.MODEL_NPZD)) for _ in range(16)]
    Y0 = torch.from_numpy(np.vstack(ys)).cuda()
    Y1 = ens.year_map(Y0, torch.empty_like(Y0)).cpu().numpy()
    assert np.all(np.isfinite(Y1))
    for m in range(16):
        m0 = float((ys[m].sum(axis=0) * p.vol).sum())
        m1 = float((Y1[5 * m:5 * m + 5].sum(axis=0) * p.vol).sum())
        assert abs(m1 - m0) <= 1e-12 * m0, m
    ens.close()


def test_adjoint_gradient_matches_central_differences(m3d, grid):
    # the 1-degree tiles do not hold their operators in shared memory, so the adjoint runs the
    # streaming sweep; checkpoint every 480 steps.  J(u) = 1/2 |M (phi(y0; u) - obs)|^2 on a
    # random 10 % of the cells, against central differences with h = 1e-6 relative
    p, _ = grid
    r = mi.rng(1410, "observations")
    ctx = m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    assert ctx.get_option(m3d.OPT_ADJOINT_PLAN) == m3d.PLAN_PERSISTENT
    u0 = mi.default_params_ndop()
    y0 = torch.from_numpy(mi.random_state(p, seed=41)).cuda()
    mask = torch.from_numpy((r.random((2, p.n)) < 0.1).astype(np.float64)).cuda()
    obs = y0 * torch.from_numpy(1.0 + 0.05 * r.standard_normal((2, p.n))).cuda()

    def J(uu):
        y1 = torch.empty_like(y0)
        ctx.year_map(y0, y1, torch.from_numpy(uu).cuda())
        return 0.5 * float(torch.sum((mask * (y1 - obs)) ** 2))

    y1 = torch.empty_like(y0)
    ctx.year_map(y0, y1, torch.from_numpy(u0).cuda())
    grad = ctx.year_adjoint(y0, torch.from_numpy(u0).cuda(), mask * mask * (y1 - obs), torch.empty_like(y0), 480)
    J0 = J(u0)
    for k in range(7):
        e = 1e-6 * u0[k]
        up, um = u0.copy(), u0.copy()
        up[k] += e
        um[k] -= e
        fd = (J(up) - J(um)) / (2 * e)
        assert abs(grad[k] - fd) <= 1e-5 * abs(fd) + 1e-9 * J0, (k, grad[k], fd)
    ctx.close()


def test_npzd_tangent_ensemble_matches_differences(m3d, grid):
    """The 16-member NPZD-DOP tangent ensemble over a few steps against central differences of
    the plain ensemble's steps (whose parity with the oracle the tests above check)."""
    p, _ = grid
    members = mi.make_ensemble(((mi.MODEL_NPZD, 16),), seed=5)
    ens = m3d.Ensemble.from_problem(p, members)
    tan = m3d.Ensemble.from_problem(p, members, tangent=True)
    ys = [mi.random_state(p, 5, seed=300 + i, scale=(4.4, 0.07, 0.07, 0.07, 0.05)) for i in range(16)]
    r = np.random.default_rng(12)
    Y = torch.from_numpy(np.vstack(ys)).cuda()
    V = torch.from_numpy(r.standard_normal((80, p.n))).cuda()
    j0, nsteps = 700, 4
    out = tan.steps(j0, nsteps, torch.cat([Y, V]), torch.empty((160, p.n), dtype=torch.float64, device="cuda"))
    jv = out[80:].cpu().numpy()
    h = 1e-6 * float(torch.linalg.norm(Y)) / float(torch.linalg.norm(V))
    yp = ens.steps(j0, nsteps, Y + h * V, torch.empty_like(Y)).cpu().numpy()
    ym = ens.steps(j0, nsteps, Y - h * V, torch.empty_like(Y)).cpu().numpy()
    fd = (yp - ym) / (2 * h)
    assert rel_err(out[:80].cpu().numpy(), ens.steps(j0, nsteps, Y, torch.empty_like(Y)).cpu().numpy()) < 1e-13
    for m in range(16):
        a = slice(5 * m, 5 * m + 5)
        assert np.abs(jv[a] - fd[a]).max() <= 1e-6 * np.abs(fd[a]).max(), m
    ens.close()
    tan.close()


def test_npzd_ensemble_adjoint_gradient_matches_differences(m3d, grid):
    """The 16-member NPZD-DOP ensemble's reverse sweep at 1 degree (checkpoint every 480 steps):
    the gradient of J = 1/2 |M (phi(Y; u) - obs)|^2 (M: a random 10 % of the cells) in a few
    parameters of two members, against central differences of the ensemble year map."""
    p, _ = grid
    members = mi.make_ensemble(((mi.MODEL_NPZD, 16),), seed=7)
    ens = m3d.Ensemble.from_problem(p, members)
    r = mi.rng(1410, "observations")
    ys = [mi.initial_state(p, 5, mi.model_initial_values(mi.MODEL_NPZD)) for _ in range(16)]
    Y0 = torch.from_numpy(np.vstack(ys)).cuda()
    mask = torch.from_numpy((r.random((80, p.n)) < 0.1).astype(np.float64)).cuda()
    Y1 = ens.year_map(Y0, torch.empty_like(Y0))
    obs = Y1 * torch.from_numpy(1.0 + 0.05 * r.standard_normal((80, p.n))).cuda()

    def J():
        y1 = ens.year_map(Y0, torch.empty_like(Y0))
        return 0.5 * float(torch.sum((mask * (y1 - obs)) ** 2))

    grads = ens.year_adjoint(Y0, mask * mask * (Y1 - obs), torch.empty_like(Y0), ckpt_every=480)
    J0 = J()
    for m, k in ((0, 0), (0, 1), (9, 12)):
        u0 = np.asarray(members[m].u, dtype=np.float64)
        e = 1e-6 * u0[k]
        vals = []
        for sgn in (1.0, -1.0):
            uu = u0.copy()
            uu[k] += sgn * e
            ens.set_params(m, uu)
            vals.append(J())
        ens.set_params(m, u0)
        fd = (vals[0] - vals[1]) / (2 * e)
        assert abs(grads[m][k] - fd) <= 1e-5 * abs(fd) + 1e-9 * J0, (m, k, grads[m][k], fd)
    ens.close()
