"""The gradient at the periodic solution (metos3d_periodic_gradient) against the oracle.

On the 6 x 4 x 4 grid the oracle's dense implicit-function gradient (pinned to central
differences of Newton-solved periodic states) is the reference.  On the 64 x 32 x 8 grid,
too large for the dense oracle, the adjoint solution lambda the library returns after a
bounded number of iterations is checked against the equation that defines it, evaluated with
the oracle's adjoint year map: the residual of P (lambda - phi_y^T lambda) = P g is the one
reported, vol^T lambda = 0, and ubar = phi_u^T lambda.
"""
import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from oracle import implicit
from oracle.newton import newton_krylov

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    return m


def oracle_periodic_state(P, y0, u, tol):
    jv = lambda y, py, v: oracle.year_tangent(P, y, v, u)[1]
    ys, rep = newton_krylov(P, y0, u, tol=tol, jv=jv, max_newton=60)
    assert rep["converged"]
    return ys


def misfit(ystar, seed=1410, frac=0.5):
    r = mi.rng(seed, "observations")
    mask = (r.random(ystar.shape) < frac).astype(np.float64)
    obs = ystar * (1.0 + 0.05 * r.standard_normal(ystar.shape))
    return mask * (ystar - obs)


def project(p, x):
    w = np.tile(p.vol, x.shape[0]).reshape(x.shape)
    return x - (np.sum(w * x) / np.sum(w * w)) * w


def test_gradient_matches_dense_oracle(m3d):
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    ystar = oracle_periodic_state(P, mi.initial_state(p), u, 3e-12)
    g = misfit(ystar)
    want = implicit.periodic_gradient(P, ystar, u, g)
    dY = implicit.periodic_state_derivative(P, ystar, u)
    terms = np.abs(dY * g.ravel()[:, None]).sum(axis=0)
    ctx = m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    lam = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    st, ubar, rep = ctx.periodic_gradient(torch.from_numpy(ystar).cuda(), torch.from_numpy(u).cuda(),
                                          torch.from_numpy(g).cuda(), lam, tol=1e-12)
    assert st == m3d.M3D_OK and rep["converged"] and rep["residual"] <= 1e-11, rep
    assert rep["forward_years"] == 1.0 and rep["reverse_sweeps"] >= rep["krylov"] + 1
    assert np.all(np.abs(ubar - want) <= 1e-8 * terms), (ubar, want)
    lam_h = lam.cpu().numpy()
    assert abs(float(np.sum(np.tile(p.vol, 2).reshape(lam_h.shape) * lam_h))) <= 1e-12 * np.abs(lam_h).sum() * p.vol.max()
    # checkpointed reverse sweeps (segments recomputed every time) give the same result, up to
    # the order in which the per-segment parameter gradients are summed
    st2, ubar2, rep2 = ctx.periodic_gradient(torch.from_numpy(ystar).cuda(), torch.from_numpy(u).cuda(),
                                             torch.from_numpy(g).cuda(), tol=1e-12, ckpt_every=240)
    assert st2 == m3d.M3D_OK and rep2["forward_years"] > 1.5
    assert np.all(np.abs(ubar2 - ubar) <= 1e-13 * terms)
    # a misfit that only changes the mass has no gradient at fixed mass
    w = np.tile(p.vol, 2).reshape(ystar.shape)
    st3, ubar3, rep3 = ctx.periodic_gradient(torch.from_numpy(ystar).cuda(), torch.from_numpy(u).cuda(),
                                             torch.from_numpy(w).cuda())
    assert st3 == m3d.M3D_OK and rep3["krylov"] == 0 and np.all(ubar3 == 0.0)
    ctx.close()


def test_adjoint_solution_and_its_residual_on_a_larger_grid(m3d):
    # 10,325 cells.  I - phi_y has a continuum of slow modes here (ventilation over centuries),
    # so GMRES reduces the residual slowly (about 1e-2 after 1000 iterations); the test runs a
    # bounded number of iterations and checks, with the oracle's adjoint year map, that what
    # the library returns is what it reports: lambda has zero mass, the residual of its
    # defining equation P (lambda - phi_y^T lambda) = P g is the reported one, it does not grow
    # with more iterations, and ubar = phi_u^T lambda.
    p = mi.make_problem("ndop_64x32x8")
    P = oracle.Problem(p)
    u = mi.default_params_ndop()
    ctx = m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    y = torch.from_numpy(mi.initial_state(p)).cuda()
    ud = torch.from_numpy(u).cuda()
    st, rep = ctx.newton_solve(y, ud, tol=1e-9, jv=m3d.JV_TANGENT)
    assert rep["converged"], rep
    ystar = y.cpu().numpy()
    g = misfit(ystar, frac=0.1)
    Pg = project(p, g)
    residuals = []
    for iters in (20, 100):
        lam = torch.empty_like(y)
        st, ubar, grep = ctx.periodic_gradient(y, ud, torch.from_numpy(g).cuda(), lam, tol=1e-12,
                                               restart=iters, max_krylov=iters)
        assert st == m3d.M3D_NOT_CONVERGED and not grep["converged"] and grep["krylov"] == iters, grep
        lam_h = lam.cpu().numpy()
        w = np.tile(p.vol, 2).reshape(lam_h.shape)
        assert abs(float(np.sum(w * lam_h))) <= 1e-12 * float(np.sum(np.abs(w * lam_h)))
        lt_phi_y, lt_phi_u = oracle.year_adjoint(P, ystar, u, lam_h)
        resid = np.linalg.norm(project(p, lam_h - lt_phi_y) - Pg) / np.linalg.norm(Pg)
        assert abs(resid - grep["residual"]) <= 1e-6 * resid, (resid, grep["residual"])
        assert np.all(np.abs(ubar - lt_phi_u) <= 1e-10 * np.abs(lt_phi_u) + 1e-12 * np.max(np.abs(lt_phi_u)))
        residuals.append(resid)
    assert residuals[1] < residuals[0] < 1.0
    ctx.close()


def test_models_without_an_adjoint_are_refused(m3d):
    p = mi.make_problem("tiny_6x4x4")
    sp = mi.MODELS[mi.MODEL_PHY]
    ctx = m3d.Context.from_problem(p, model=mi.MODEL_PHY, ntracer=len(sp.tracers), nparam=len(sp.params))
    y = torch.from_numpy(mi.initial_state(p, 3, mi.model_initial_values(mi.MODEL_PHY))).cuda()
    with pytest.raises(m3d.Metos3dError) as e:
        ctx.periodic_gradient(y, torch.from_numpy(mi.default_params(mi.MODEL_PHY)).cuda(), torch.zeros_like(y))
    assert e.value.status == m3d.M3D_ERR_UNSUPPORTED
    ctx.close()
