"""Single contexts of the N, PO4-DOP-PHY and NPZD-DOP models (run by a one-member ensemble inside
the library) through the C ABI: year map and step against the oracle, host and device entry
points, the ensemble they use, and the paper's periodic solve (Section 7 compares spin-up and
Newton's method on PO4-DOP-PHY) on a small grid.
"""
import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from tests._util import normwise_err, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MODELS = [mi.MODEL_N, mi.MODEL_PHY, mi.MODEL_NPZD]


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def context(m3d, p, model):
    sp = mi.MODELS[model]
    return m3d.Context.from_problem(p, model=model, ntracer=len(sp.tracers), nparam=len(sp.params))


@pytest.mark.parametrize("model", MODELS)
def test_year_map_and_step_match_oracle(m3d, model):
    p = mi.make_problem("ndop_64x32x8")
    P = oracle.Problem(p)
    ntr = len(mi.MODELS[model].tracers)
    u = mi.default_params(model)
    y0 = mi.initial_state(p, ntr, mi.model_initial_values(model))
    ctx = context(m3d, p, model)
    y1 = ctx.year_map(torch.from_numpy(y0).cuda(), torch.empty((ntr, p.n), dtype=torch.float64, device="cuda"),
                      torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(y1, oracle.year_map(P, y0, u, model=model)) <= 1e-10
    ys = mi.random_state(p, ntr, seed=17, scale=tuple(2.0 * v + 0.05 for v in mi.model_initial_values(model)))
    s1 = ctx.step(613, torch.from_numpy(ys).cuda(), torch.empty((ntr, p.n), dtype=torch.float64, device="cuda"),
                  torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(s1, oracle.step(P, 613, ys, u, model=model)) <= 1e-13
    # the host entry point and the ensemble the context runs give the same bits
    assert np.array_equal(ctx.year_map_host(y0, u), y1)
    ens = m3d.Ensemble.from_problem(p, [mi.Member(model, u)])
    Y = torch.from_numpy(y0).cuda()
    assert np.array_equal(ens.year_map(Y, torch.empty_like(Y)).cpu().numpy(), y1)
    ens.close()
    # the plan options belong to the tiled kernels
    with pytest.raises(m3d.Metos3dError) as ei:
        ctx.set_option(m3d.OPT_YEAR_PLAN, m3d.PLAN_RESIDENT)
    assert ei.value.status == m3d.M3D_ERR_UNSUPPORTED
    ctx.close()


def test_phy_periodic_solution_newton_against_spinup(m3d):
    # PO4-DOP-PHY, the paper's Section 7 model: Newton-Krylov (finite differences) reaches
    # ||phi(y) - y|| < 1e-8; the oracle's year map confirms the residual; mass is kept; a
    # spin-up from the same start decreases its residual but stays far from the tolerance
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = mi.default_params(mi.MODEL_PHY)
    y0 = mi.initial_state(p, 3, mi.model_initial_values(mi.MODEL_PHY))
    ctx = context(m3d, p, mi.MODEL_PHY)
    y = torch.from_numpy(y0).cuda()
    st, rep = ctx.newton_solve(y, torch.from_numpy(u).cuda(), tol=1e-8)
    assert rep["converged"] and rep["residual"] < 1e-8
    ys = y.cpu().numpy()
    r_oracle = float(np.linalg.norm(oracle.year_map(P, ys, u, model=mi.MODEL_PHY) - ys))
    assert r_oracle < 1e-7
    m0 = float((y0.sum(axis=0) * p.vol).sum())
    assert abs(float((ys.sum(axis=0) * p.vol).sum()) - m0) <= 1e-10 * m0
    ysp = torch.from_numpy(y0).cuda()
    res = ctx.spinup(ysp, torch.from_numpy(u).cuda(), 50)
    assert res.size == 50 and res[-1] < res[0] and res[-1] > 1e-8
    ctx.close()


@pytest.mark.parametrize("model", [mi.MODEL_N, mi.MODEL_PHY, mi.MODEL_NPZD])
def test_single_context_tangent_of_every_model(m3d, model):
    """metos3d_year_tangent of an N, PO4-DOP-PHY or NPZD-DOP context (a one-member tangent
    ensemble) against the oracle's tangent year map; Newton-Krylov with those products."""
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    ntr = len(mi.MODELS[model].tracers)
    u = np.asarray(mi.default_params(model), dtype=np.float64)
    ctx = context(m3d, p, model)
    y = mi.initial_state(p, ntr, mi.model_initial_values(model)) * (0.5 + np.random.default_rng(1).random((ntr, p.n)))
    v = np.random.default_rng(2).standard_normal((ntr, p.n))
    phi = torch.empty((ntr, p.n), dtype=torch.float64, device="cuda")
    jv = torch.empty_like(phi)
    ctx.year_tangent(cuda(y), cuda(v), cuda(u), phi, jv)
    ctx.sync()
    want_phi, want_jv = oracle.year_tangent(P, y, v, u, model=model)
    assert rel_err(phi.cpu().numpy(), want_phi) < 1e-10
    assert normwise_err(jv.cpu().numpy(), want_jv) < 1e-10
    if model == mi.MODEL_NPZD:
        # (NPZD-DOP's periodic solve from its constant start takes hundreds of Krylov
        # iterations per Newton step; the solver itself is the same for every model)
        ctx.close()
        return
    y0 = mi.initial_state(p, ntr, mi.model_initial_values(model))
    yN = cuda(y0)
    st, rep = ctx.newton_solve(yN, cuda(u), tol=1e-8, jv=m3d.JV_TANGENT)
    assert st == m3d.M3D_OK and rep["tangent_maps"] > 0, rep
    got = yN.cpu().numpy()
    assert np.linalg.norm((oracle.year_map(P, got, u, model=model) - got).ravel()) < 2e-8
    ctx.close()


@pytest.mark.parametrize("model", [mi.MODEL_N, mi.MODEL_PHY, mi.MODEL_NPZD])
def test_single_context_adjoint_of_every_model(m3d, model):
    """metos3d_year_adjoint of an N, PO4-DOP-PHY or NPZD-DOP context (the reverse sweep of its
    one-member ensemble) against the oracle's adjoint year map."""
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    ntr = len(mi.MODELS[model].tracers)
    u = np.asarray(mi.default_params(model), dtype=np.float64)
    ctx = context(m3d, p, model)
    y = mi.initial_state(p, ntr, mi.model_initial_values(model)) * (0.5 + np.random.default_rng(3).random((ntr, p.n)))
    wbar = np.random.default_rng(4).standard_normal((ntr, p.n))
    yb0 = torch.empty((ntr, p.n), dtype=torch.float64, device="cuda")
    ubar = ctx.year_adjoint(cuda(y), cuda(u), cuda(wbar), yb0, 240)
    want_y, want_u = oracle.year_adjoint(P, y, u, wbar, model=model)
    assert normwise_err(yb0.cpu().numpy(), want_y) < 1e-10
    assert np.abs(ubar - want_u).max() <= 1e-9 * np.abs(want_u).max(), (ubar, want_u)
    ctx.close()
