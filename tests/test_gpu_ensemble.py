"""Parity of the batched ensemble (metos3d_ensemble_*, through the C ABI) with the CPU oracle.

The oracle of an ensemble is every member's own year map (members share only the transport).
Tolerance as for the single year map: 1e-10 in max_i |g_i - o_i| / max(|o_i|, 1e-6 max|o|) per
model year, per member, in FP64.
"""
import os

import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from tests._util import normwise_err, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

YEAR_TOL = 1e-10
STEP_TOL = 1e-12

# every model, several groups of 32 lanes (W = 2*1 + 3*2 + 2*3 + 5*5 = 39: two groups)
SMALL_MIX = ((mi.MODEL_N, 2), (mi.MODEL_NDOP, 3), (mi.MODEL_PHY, 2), (mi.MODEL_NPZD, 5))


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    oracle.set_threads(min(16, os.cpu_count() or 1))
    yield m
    oracle.set_threads(1)


_problems = {}


def problem(name):
    if name not in _problems:
        p = mi.make_problem(name)
        _problems[name] = (p, oracle.Problem(p))
    return _problems[name]


def initial_states(prob, members, seed=None):
    """Member states: the models' constant initial values, or seeded positive fields."""
    out = []
    for i, m in enumerate(members):
        vals = mi.model_initial_values(m.model)
        if seed is None:
            out.append(mi.initial_state(prob, m.ntracer, vals))
        else:
            y = mi.random_state(prob, m.ntracer, seed=seed + i, scale=tuple(2.0 * v + 0.05 for v in vals))
            out.append(y)
    return out


def stack(states):
    return torch.from_numpy(np.ascontiguousarray(np.vstack(states))).cuda()


def split(ens, Y):
    Yh = Y.cpu().numpy()
    return [Yh[ens.offsets[m]:ens.offsets[m + 1]] for m in range(ens.nmember)]


def test_year_map_matches_oracle_every_model(m3d):
    p, P = problem("ndop_64x32x8")
    members = mi.make_ensemble(SMALL_MIX, seed=11)
    ens = m3d.Ensemble.from_problem(p, members)
    assert ens.width == 39 and ens.ngroup == 2
    ys = initial_states(p, members)
    Y1 = ens.year_map(stack(ys), torch.empty((ens.width, p.n), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert ens.last_launch_count() == p.nstep + 2
    want = oracle.ensemble_year_map(P, ys, members)
    for m, (g, o) in enumerate(zip(split(ens, Y1), want)):
        assert rel_err(g, o) <= YEAR_TOL, (m, members[m].model, rel_err(g, o))
    ens.close()


def test_year_map_conserves_each_members_mass(m3d):
    p, _ = problem("ndop_64x32x8")
    members = mi.make_ensemble(SMALL_MIX, seed=12)
    ens = m3d.Ensemble.from_problem(p, members)
    ys = initial_states(p, members, seed=40)
    Y1 = ens.year_map(stack(ys), torch.empty((ens.width, p.n), dtype=torch.float64, device="cuda"))
    for y0, y1 in zip(ys, split(ens, Y1)):
        m0 = float((y0.sum(axis=0) * p.vol).sum())
        m1 = float((y1.sum(axis=0) * p.vol).sum())
        assert abs(m1 - m0) <= 1e-12 * m0
        assert np.all(np.isfinite(y1))
    ens.close()


def test_full_mix_steps_match_oracle_on_the_full_grid(m3d):
    # the 64-member ensemble (16 N, 32 N-DOP, 16 NPZD-DOP; five full groups) on 128 x 64 x 15,
    # a ragged sample of steps across a month boundary, varying states
    p, P = problem("ndop_128x64x15")
    members = mi.make_ensemble()
    ens = m3d.Ensemble.from_problem(p, members)
    assert ens.width == 160 and ens.ngroup == 5
    ys = initial_states(p, members, seed=7)
    j0, nsteps = 235, 13
    Y1 = ens.steps(j0, nsteps, stack(ys), torch.empty((ens.width, p.n), dtype=torch.float64, device="cuda"))
    want = oracle.ensemble_steps(P, j0, nsteps, ys, members)
    for m, (g, o) in enumerate(zip(split(ens, Y1), want)):
        assert rel_err(g, o) <= STEP_TOL, (m, members[m].model, rel_err(g, o))
    ens.close()


@pytest.mark.parametrize("nsub", [2, 8])
def test_internal_model_steps_match_oracle(m3d, nsub):
    p, P = problem("ndop_64x32x8")
    members = mi.make_ensemble(SMALL_MIX, seed=13)
    ens = m3d.Ensemble.from_problem(p, members, nsub=nsub)
    ys = initial_states(p, members, seed=3)
    Y1 = ens.steps(1000, 40, stack(ys), torch.empty((ens.width, p.n), dtype=torch.float64, device="cuda"))
    r = np.random.default_rng(0)
    for m, (g, y, mem) in enumerate(zip(split(ens, Y1), ys, members)):
        o = oracle.steps(P, 1000, 40, y, mem.u, model=mem.model, nsub=nsub)
        # The two sides round differently (fused multiply-adds, one shared division), and
        # 40 ocean steps of a grazing model from random states amplify rounding-level input
        # differences by up to ~1e4.  The bar is the oracle's own response to a perturbation
        # of its input by a few units in the last place, with headroom, and never above the
        # per-year 1e-10.
        o_pert = oracle.steps(P, 1000, 40, y * (1.0 + 4e-16 * r.standard_normal(y.shape)), mem.u,
                              model=mem.model, nsub=nsub)
        bar = min(1e-10, max(STEP_TOL, 20.0 * rel_err(o_pert, o)))
        assert rel_err(g, o) <= bar, (m, mem.model, rel_err(g, o), bar)
    ens.close()


def test_results_do_not_depend_on_tiling_or_neighbours(m3d):
    # each lane runs the same arithmetic whatever the tiling and the other members
    p, _ = problem("ndop_64x32x8")
    members = mi.make_ensemble(SMALL_MIX, seed=14)
    ens = m3d.Ensemble.from_problem(p, members)
    Y0 = stack(initial_states(p, members, seed=5))
    ref = ens.steps(700, 25, Y0, torch.empty_like(Y0)).clone()
    for cpb, nw in ((1, 4), (2, 16), (8, 8), (32, 4)):
        ens.set_tiling(cpb, nw)
        assert ens.get_tiling() == (cpb, nw)
        assert torch.equal(ens.steps(700, 25, Y0, torch.empty_like(Y0)), ref)
    cpb, nw, ms = ens.autotune(Y0, nsteps=5)
    assert ens.get_tiling() == (cpb, nw) and ms > 0.0
    assert torch.equal(ens.steps(700, 25, Y0, torch.empty_like(Y0)), ref)
    # one member alone gives bit for bit the same result
    for m in (0, 3, 7, len(members) - 1):
        alone = m3d.Ensemble.from_problem(p, [members[m]])
        ym = Y0[ens.offsets[m]:ens.offsets[m + 1]].contiguous()
        got = alone.steps(700, 25, ym, torch.empty_like(ym))
        assert torch.equal(got, ref[ens.offsets[m]:ens.offsets[m + 1]]), m
        alone.close()
    ens.close()


def test_year_graph_equals_single_launches(m3d):
    p, _ = problem("ndop_64x32x8")
    members = mi.make_ensemble(SMALL_MIX, seed=15)
    ens = m3d.Ensemble.from_problem(p, members)
    Y0 = stack(initial_states(p, members, seed=9))
    a = ens.year_map(Y0, torch.empty_like(Y0)).clone()
    b = ens.steps(0, p.nstep, Y0, torch.empty_like(Y0))
    assert torch.equal(a, b)
    # in place
    Y = Y0.clone()
    ens.year_map(Y, Y)
    assert torch.equal(Y, a)
    ens.close()


def test_set_params_takes_effect(m3d):
    p, P = problem("ndop_64x32x8")
    members = mi.make_ensemble(((mi.MODEL_NDOP, 2), (mi.MODEL_NPZD, 1)), seed=16)
    ens = m3d.Ensemble.from_problem(p, members)
    ys = initial_states(p, members, seed=21)
    Y0 = stack(ys)
    before = split(ens, ens.steps(0, 30, Y0, torch.empty_like(Y0)))
    u_new = members[2].u * 1.3
    u_new[6] = min(u_new[6], 1.0)
    ens.set_params(2, u_new)
    after = split(ens, ens.steps(0, 30, Y0, torch.empty_like(Y0)))
    assert np.array_equal(before[0], after[0]) and not np.array_equal(before[2], after[2])
    o = oracle.steps(P, 0, 30, ys[2], u_new, model=mi.MODEL_NPZD)
    assert rel_err(after[2], o) <= STEP_TOL
    ens.close()


def test_ndop_member_matches_single_context(m3d):
    # an N-DOP member of an ensemble and the single-context year map (resident kernel) agree
    p, _ = problem("ndop_64x32x8")
    members = mi.make_ensemble(((mi.MODEL_NDOP, 1), (mi.MODEL_NPZD, 1)), seed=17)
    ens = m3d.Ensemble.from_problem(p, members)
    ys = initial_states(p, members, seed=33)
    Y1 = ens.year_map(stack(ys), torch.empty((ens.width, p.n), dtype=torch.float64, device="cuda"))
    ctx = m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    y0 = torch.from_numpy(ys[0]).cuda()
    y1 = ctx.year_map(y0, torch.empty_like(y0), torch.from_numpy(members[0].u).cuda())
    assert rel_err(split(ens, Y1)[0], y1.cpu().numpy()) <= 1e-12
    ctx.close()
    ens.close()


def test_rejects_oversized_tiling(m3d):
    p, _ = problem("ndop_128x64x15")
    ens = m3d.Ensemble.from_problem(p, mi.make_ensemble(((mi.MODEL_N, 1),), seed=1))
    with pytest.raises(m3d.Metos3dError) as ei:
        ens.set_tiling(4000, 16)
    assert ei.value.status == m3d.M3D_ERR_ARG
    ens.close()


def tangent_sensitivity(P, y, v, mem, nsub, jv):
    """How much the oracle's own phi'(y) v moves (normwise) when y moves by a rounding-level
    1e-14 relative: two correct FP64 evaluations whose trajectories differ by rounding cannot
    agree better.  Tiny for the transport-dominated models; NPZD-DOP's predator-prey
    dynamics amplify it to 1e-10 .. 1e-8 on these grids."""
    r = np.random.default_rng(77)
    y2 = y * (1.0 + 1e-14 * r.standard_normal(y.shape))
    _, jv2 = oracle.year_tangent(P, y2, v, mem.u, model=mem.model, nsub=nsub)
    return normwise_err(jv2, jv)


def adjoint_sensitivity(P, y, wb, mem, yb, ub):
    """The same for the oracle's adjoint year map (state cotangent, parameter gradient)."""
    r = np.random.default_rng(78)
    y2 = y * (1.0 + 1e-14 * r.standard_normal(y.shape))
    yb2, ub2 = oracle.year_adjoint(P, y2, mem.u, wb, model=mem.model)
    return normwise_err(yb2, yb), float(np.abs(ub2 - ub).max() / np.abs(ub).max())


@pytest.mark.parametrize("grid,nsub", [("tiny_6x4x4", 1), ("tiny_6x4x4", 3), ("ndop_64x32x8", 1)])
def test_tangent_ensemble_matches_oracle_tangent(m3d, grid, nsub):
    """A tangent ensemble (every model, several lane groups) returns each member's phi(y) and
    phi'(y) v, checked against the oracle's tangent year map of that member."""
    p, P = problem(grid)
    members = mi.make_ensemble(SMALL_MIX, seed=13)
    ens = m3d.Ensemble.from_problem(p, members, tangent=True, nsub=nsub)
    W = sum(m.ntracer for m in members)
    assert ens.width == 2 * W
    ys = initial_states(p, members, seed=40)
    r = np.random.default_rng(5)
    vs = [r.standard_normal(y.shape) for y in ys]
    Y = stack(ys + vs)
    Y1 = ens.year_map(Y, torch.empty_like(Y)).cpu().numpy()
    for m, (y, v, mem) in enumerate(zip(ys, vs, members)):
        a, b = ens.offsets[m], ens.offsets[m + 1]
        want_phi, want_jv = oracle.year_tangent(P, y, v, mem.u, model=mem.model, nsub=nsub)
        assert rel_err(Y1[a:b], want_phi) < YEAR_TOL, m
        # a signed perturbation field: normwise, within the tangent's own condition
        tol = max(YEAR_TOL, 10.0 * tangent_sensitivity(P, y, v, mem, nsub, want_jv))
        assert normwise_err(Y1[W + a:W + b], want_jv) < tol, (m, tol)
    ens.close()


@pytest.mark.parametrize("grid,ckpt", [("tiny_6x4x4", 240), ("tiny_6x4x4", 7), ("ndop_64x32x8", 480)])
def test_ensemble_adjoint_matches_oracle_adjoint(m3d, grid, ckpt):
    """The reverse sweep of a mixed ensemble (every model) against each member's own adjoint
    year map in the oracle: the state cotangent normwise, the parameter gradient relative to
    its largest entry."""
    p, P = problem(grid)
    members = mi.make_ensemble(SMALL_MIX, seed=17)
    ens = m3d.Ensemble.from_problem(p, members)
    ys = initial_states(p, members, seed=60)
    r = np.random.default_rng(9)
    wbars = [r.standard_normal(y.shape) for y in ys]
    Yb0 = torch.empty((ens.width, p.n), dtype=torch.float64, device="cuda")
    ubs = ens.year_adjoint(stack(ys), stack(wbars), Yb0, ckpt_every=ckpt)
    Yb0 = Yb0.cpu().numpy()
    for m, (y, wb, mem) in enumerate(zip(ys, wbars, members)):
        a, b = ens.offsets[m], ens.offsets[m + 1]
        want_y, want_u = oracle.year_adjoint(P, y, mem.u, wb, model=mem.model)
        sy, su = adjoint_sensitivity(P, y, wb, mem, want_y, want_u)
        assert normwise_err(Yb0[a:b], want_y) < max(1e-10, 10.0 * sy), (m, sy)
        assert np.abs(ubs[m] - want_u).max() <= max(1e-9, 10.0 * su) * np.abs(want_u).max(), (m, ubs[m], want_u)
    ens.close()


@pytest.mark.parametrize("jv", ["tangent", "fd"])
def test_ensemble_newton_every_member_periodic(m3d, jv):
    """Every member's periodic solve at once (one year map of the tangent ensemble per Krylov
    iteration of all members): each member reaches ||phi(y) - y|| < 1e-8 by its own oracle
    year map, keeps its mass, and matches the oracle's Newton-Krylov of that member alone."""
    from oracle import newton as on
    import math
    p, P = problem("tiny_6x4x4")
    # N, PO4-DOP and PO4-DOP-PHY members (NPZD-DOP's periodic solve from its constant start
    # takes hundreds of Krylov iterations per Newton step in the oracle as on the GPU)
    members = mi.make_ensemble(((mi.MODEL_N, 2), (mi.MODEL_NDOP, 3), (mi.MODEL_PHY, 2)), seed=23)
    ens = m3d.Ensemble.from_problem(p, members)
    tan = m3d.Ensemble.from_problem(p, members, tangent=True) if jv == "tangent" else None
    ys = initial_states(p, members)
    Y = stack(ys)
    st, reps = ens.newton_solve(Y, p.vol, tangent_ensemble=tan, tol=1e-8,
                                jv=m3d.JV_TANGENT if jv == "tangent" else m3d.JV_FD)
    assert st == m3d.M3D_OK, [r["residual"] for r in reps]
    got = Y.cpu().numpy()
    for m, (y0, mem) in enumerate(zip(ys, members)):
        a, b = ens.offsets[m], ens.offsets[m + 1]
        gm = got[a:b]
        assert reps[m]["converged"] and reps[m]["residual"] < 1e-8
        assert np.linalg.norm((oracle.year_map(P, gm, mem.u, model=mem.model) - gm).ravel()) < 2e-8, m
        m0 = math.fsum((p.vol * y0).ravel())
        assert abs(math.fsum((p.vol * gm).ravel()) / m0 - 1) < 1e-12, m
        want, _ = on.newton_krylov(P, y0, mem.u, tol=1e-8, model=mem.model)
        assert np.abs(gm - want).max() / np.abs(want).max() < 1e-6, m
    ens.close()
    if tan:
        tan.close()


def test_ensemble_newton_line_search_through_trials_that_overflow(m3d):
    """Two NPZD-DOP members in lockstep (phytoplankton x 10 and x 1 from the constant start,
    three Krylov iterations per step, tangent products): full steps of both overflow the year
    map and are cut to a tenth, each member on its own trials.  Every member's trials,
    residuals and state match the oracle's Newton of that member alone."""
    from oracle import newton as on
    p, P = problem("tiny_6x4x4")
    u = np.asarray(mi.default_params(mi.MODEL_NPZD), dtype=np.float64)
    members = [mi.Member(mi.MODEL_NPZD, u), mi.Member(mi.MODEL_NPZD, u)]
    ens = m3d.Ensemble.from_problem(p, members)
    tan = m3d.Ensemble.from_problem(p, members, tangent=True)
    base = mi.initial_state(p, 5, mi.model_initial_values(mi.MODEL_NPZD))
    ys = [base * np.array((1.0, sp, 1.0, 1.0, 1.0))[:, None] for sp in (10.0, 1.0)]
    Y = stack(ys)
    st, reps = ens.newton_solve(Y, p.vol, tangent_ensemble=tan, tol=1e-8, jv=m3d.JV_TANGENT, max_newton=4,
                                restart=3, max_krylov=3)
    assert st == m3d.M3D_NOT_CONVERGED
    got = split(ens, Y)

    def tangent(yy, py, v):
        return oracle.year_tangent(P, yy, v, u, model=mi.MODEL_NPZD)[1]

    for m in range(2):
        want, orep = on.newton_krylov(P, ys[m], u, tol=1e-8, max_newton=4, restart=3, max_krylov=3,
                                      model=mi.MODEL_NPZD, jv=tangent)
        assert orep["trials"][0][:2] == [1.0, 0.1], orep["trials"]     # the full step overflowed
        assert not reps[m]["line_search_failed"]
        assert reps[m]["krylov"] == orep["krylov"], m
        assert [len(t) for t in reps[m]["trials"]] == [len(t) for t in orep["trials"]], m
        for k in range(len(orep["trials"])):
            assert np.allclose(reps[m]["trials"][k], orep["trials"][k], rtol=1e-6, atol=0), (m, k)
        assert np.allclose(reps[m]["residuals"], orep["residuals"], rtol=1e-5, atol=0), m
        assert np.isfinite(got[m]).all() and np.abs(got[m] - want).max() / np.abs(want).max() < 1e-5, m
    ens.close()
    tan.close()
