"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerance: the year map must stay within 1e-10 of the oracle in the relative measure
max_i |g_i - o_i| / max(|o_i|, 1e-6 max|o|) per model year, in FP64.  The two sides sum
every row in the same order; they differ only in how the month interpolation is rounded
and in fused multiply-adds, so single steps agree to about 1e-15.
"""
import math
import os

import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from tests._util import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

YEAR_TOL = 1e-10
STEP_TOL = 1e-13


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    return m


_problems = {}


def problem(name):
    if name not in _problems:
        p = mi.make_problem(name)
        _problems[name] = (p, oracle.Problem(p))
    return _problems[name]


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ctx_for(m3d, prob, **kw):
    kw.setdefault("model", m3d.MODEL_NDOP)
    kw.setdefault("ntracer", 2)
    kw.setdefault("nparam", 7)
    return m3d.Context.from_problem(prob, **kw)


# ------------------------------------------------------------------ q alone (Section 5.2 interface)
@pytest.mark.parametrize("nl", [1, 2, 3, 5, 8, 15, 23])
@pytest.mark.parametrize("nsub", [1, 8])
def test_bgc_matches_oracle(m3d, nl, nsub):
    r = np.random.default_rng(100 * nl + nsub)
    h = np.array([50.0, 70, 100, 140, 190, 240, 290, 340, 390, 440, 490, 540, 590, 640, 690] + [700.0] * 8)[:nl]
    d = np.cumsum(h) - 0.5 * h
    for _ in range(5):
        u = mi.default_params_ndop() * r.uniform(0.5, 1.5, 7)
        y = r.uniform(0.0, 3.0, (2, nl))
        insol = r.uniform(0.0, 500.0)
        want = oracle.bgc(y, h, d, u, insol=insol, nsub=nsub)
        got = m3d.bgc(y, h, d, u, insol=insol, nsub=nsub)
        tol = 16 * nsub * np.finfo(float).eps * np.abs(y).max() + 1e-300
        assert np.abs(got - want).max() <= tol


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("name", ["tiny_4x3x3", "tiny_6x4x4", "ndop_64x32x8"])
def test_step_matches_oracle(m3d, name):
    p, P = problem(name)
    u = mi.default_params_ndop()
    ctx = ctx_for(m3d, p)
    y = mi.random_state(p)
    yd, ud = cuda(y), cuda(u)
    out = torch.empty_like(yd)
    for j in (0, 1, 119, 120, 121, 1439, 2879):
        ctx.step(j, yd, out, ud)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), oracle.step(P, j, y, u)) < STEP_TOL, j
    ctx.close()


def test_step_transport_only_many_tracers(m3d):
    p, P = problem("tiny_6x4x4")
    for ntr in (1, 3, 8):
        ctx = ctx_for(m3d, p, model=m3d.MODEL_NONE, ntracer=ntr, nparam=0)
        y = mi.random_state(p, ntracer=ntr)
        yd = cuda(y)
        out = torch.empty_like(yd)
        ctx.step(777, yd, out, None)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), oracle.step(P, 777, y, np.zeros(0), model=oracle.MODEL_NONE)) < STEP_TOL
        ctx.close()


# ------------------------------------------------------------------ year maps
PLANS = {"resident": 2, "persistent": 0, "graph": 1}
LAUNCHES = {"resident": 4, "persistent": 2, "graph": 2881}


@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("name,nsub", [("tiny_4x3x3", 1), ("tiny_6x4x4", 8), ("ndop_64x32x8", 1)])
def test_year_map_matches_oracle(m3d, name, nsub, plan):
    p, P = problem(name)
    u = mi.default_params_ndop()
    ctx = ctx_for(m3d, p, nsub=nsub)
    assert ctx.get_option(m3d.OPT_YEAR_PLAN) == m3d.PLAN_RESIDENT      # the default where it fits
    ctx.set_option(m3d.OPT_YEAR_PLAN, PLANS[plan])
    y0 = mi.initial_state(p)
    yd, ud = cuda(y0), cuda(u)
    y1 = torch.empty_like(yd)
    ctx.year_map(yd, y1, ud)
    ctx.sync()
    got = y1.cpu().numpy()
    want = oracle.year_map(P, y0, u, nsub=nsub)
    assert rel_err(got, want) < YEAR_TOL
    assert ctx.last_launch_count() == LAUNCHES[plan]
    # mass is conserved on the device too (Section 3 matrices conserve V^T y; q is column-conservative)
    m0 = math.fsum((p.vol * y0).ravel())
    assert abs(ctx.mass(y1) - m0) / m0 < 1e-12
    ctx.close()


def test_year_map_paper_grid_matches_oracle(m3d):
    """The 128 x 64 x 15 grid (52749 cells, the size of Section 7) in the benchmark's configuration."""
    p, P = problem("ndop_128x64x15")
    u = mi.default_params_ndop()
    ctx = ctx_for(m3d, p)
    y0 = mi.initial_state(p)
    yd, ud = cuda(y0), cuda(u)
    y1 = torch.empty_like(yd)
    ctx.year_map(yd, y1, ud)
    torch.cuda.synchronize()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        want = oracle.year_map(P, y0, u)
    finally:
        oracle.set_threads(1)
    assert rel_err(y1.cpu().numpy(), want) < YEAR_TOL
    ctx.close()


@pytest.mark.parametrize("name", ["ndop_64x32x8", "ndop_128x64x15"])
def test_all_plans_agree_bitwise(m3d, name):
    """All plans run the same per-tile arithmetic in the same order: identical results, in
    the dense and in the Thomas form of the implicit part."""
    p, _ = problem(name)
    u = cuda(mi.default_params_ndop())
    y0 = cuda(mi.random_state(p))
    ctx = ctx_for(m3d, p)
    ctx.set_option(m3d.OPT_IMPLICIT_FORM, m3d.IMPLICIT_DENSE)
    out = {}
    for plan, code in PLANS.items():
        ctx.set_option(m3d.OPT_YEAR_PLAN, code)
        out[plan] = torch.empty_like(y0)
        ctx.year_map(y0, out[plan], u)
    # the resident kernel interpolating every explicit entry itself, instead of streaming the
    # per-step operators built at init with the same fused multiply-add
    ctx.set_option(m3d.OPT_YEAR_PLAN, m3d.PLAN_RESIDENT)
    assert ctx.get_option(m3d.OPT_STEP_OPERATORS) == 1
    ctx.set_option(m3d.OPT_STEP_OPERATORS, 0)
    out["resident_interpolating"] = torch.empty_like(y0)
    ctx.year_map(y0, out["resident_interpolating"], u)
    ctx.sync()
    assert torch.equal(out["resident"], out["graph"])
    assert torch.equal(out["persistent"], out["graph"])
    assert torch.equal(out["resident_interpolating"], out["graph"])
    # the Thomas form: resident chains with factors in shared memory, and the streaming
    # kernels' chains reading them from global memory, blend in the same order
    ctx.set_option(m3d.OPT_IMPLICIT_FORM, m3d.IMPLICIT_TRIDIAGONAL)
    tri = {}
    for plan, code in PLANS.items():
        ctx.set_option(m3d.OPT_YEAR_PLAN, code)
        tri[plan] = torch.empty_like(y0)
        ctx.year_map(y0, tri[plan], u)
    ctx.sync()
    assert torch.equal(tri["resident"], tri["graph"])
    assert torch.equal(tri["persistent"], tri["graph"])
    assert not torch.equal(tri["graph"], out["graph"])      # the two forms differ in rounding
    ctx.close()


@pytest.mark.parametrize("name", ["tiny_6x4x4", "ndop_64x32x8", "ndop_128x64x15"])
def test_step_operators_match_in_kernel_interpolation(m3d, name):
    """Per-step explicit operators (nstep x slot-lanes doubles, built once) against the kernel
    interpolating the monthly matrices itself: bit-identical year maps in the tridiagonal
    form; the option reports and releases its memory."""
    p, _ = problem(name)
    u = cuda(mi.default_params_ndop())
    y0 = cuda(mi.random_state(p))
    ctx = ctx_for(m3d, p)
    assert ctx.get_option(m3d.OPT_IMPLICIT_FORM) == m3d.IMPLICIT_TRIDIAGONAL
    assert ctx.get_option(m3d.OPT_STEP_OPERATORS) == 1
    nbytes = ctx.get_option(m3d.OPT_STEP_OPERATOR_BYTES)
    assert nbytes > 0 and nbytes % (8 * 32 * p.nstep) == 0
    assert nbytes >= 8 * p.nnz * p.nstep                           # at least one value per entry and step
    streamed, interpolated = torch.empty_like(y0), torch.empty_like(y0)
    ctx.year_map(y0, streamed, u)
    ctx.set_option(m3d.OPT_STEP_OPERATORS, 0)
    assert ctx.get_option(m3d.OPT_STEP_OPERATORS) == 0 and ctx.get_option(m3d.OPT_STEP_OPERATOR_BYTES) == 0
    ctx.year_map(y0, interpolated, u)
    ctx.sync()
    assert torch.equal(streamed, interpolated)
    ctx.set_option(m3d.OPT_STEP_OPERATORS, 1)
    assert ctx.get_option(m3d.OPT_STEP_OPERATOR_BYTES) == nbytes
    again = torch.empty_like(y0)
    ctx.year_map(y0, again, u)
    ctx.sync()
    assert torch.equal(again, streamed)
    with pytest.raises(m3d.Metos3dError) as e:
        ctx.set_option(m3d.OPT_STEP_OPERATORS, 2)
    assert e.value.status == m3d.M3D_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("name", ["ndop_64x32x8", "ndop_128x64x15"])
def test_tridiagonal_implicit_form_matches_dense(m3d, name):
    """The synthetic implicit blocks are inverses of tridiagonal diffusion matrices: the
    Thomas form is detected and agrees with the dense interpolated product to rounding."""
    p, _ = problem(name)
    u = cuda(mi.default_params_ndop())
    y0 = cuda(mi.random_state(p))
    ctx = ctx_for(m3d, p)
    assert ctx.get_option(m3d.OPT_IMPLICIT_FORM) == m3d.IMPLICIT_TRIDIAGONAL
    tri = torch.empty_like(y0)
    dense = torch.empty_like(y0)
    ctx.year_map(y0, tri, u)
    ctx.set_option(m3d.OPT_IMPLICIT_FORM, m3d.IMPLICIT_DENSE)
    ctx.year_map(y0, dense, u)
    ctx.sync()
    assert rel_err(tri.cpu().numpy(), dense.cpu().numpy()) < 1e-12
    ctx.close()


def test_general_dense_blocks_fall_back_to_dense_form(m3d):
    """Implicit blocks that are not inverses of tridiagonal matrices keep the dense form."""
    import copy
    p0, _ = problem("tiny_6x4x4")
    p = copy.copy(p0)
    r = np.random.default_rng(3)
    p.imp_blk = p0.imp_blk * (1.0 + 0.05 * r.random(p0.imp_blk.shape))
    P = oracle.Problem(p)
    ctx = ctx_for(m3d, p)
    assert ctx.get_option(m3d.OPT_IMPLICIT_FORM) == m3d.IMPLICIT_DENSE
    with pytest.raises(m3d.Metos3dError):
        ctx.set_option(m3d.OPT_IMPLICIT_FORM, m3d.IMPLICIT_TRIDIAGONAL)
    u_h = mi.default_params_ndop()
    y0_h = mi.initial_state(p)
    y1 = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    ctx.year_map(cuda(y0_h), y1, cuda(u_h))
    ctx.sync()
    assert rel_err(y1.cpu().numpy(), oracle.year_map(P, y0_h, u_h)) < YEAR_TOL
    ctx.close()


def test_persistent_wait_timeout_is_reported_and_recoverable(m3d):
    """A tile that never announces its progress makes its neighbours' bounded waits run out:
    the kernel stops, metos3d_sync reports M3D_ERR_TIMEOUT, and the context stays usable."""
    p, P = problem("ndop_64x32x8")
    u_h = mi.default_params_ndop()
    u = cuda(u_h)
    y0_h = mi.initial_state(p)
    y0 = cuda(y0_h)
    y1 = torch.empty_like(y0)
    ctx = ctx_for(m3d, p)
    assert ctx.get_option(m3d.OPT_NTILES) > 1
    ctx.set_option(m3d.OPT_WAIT_TIMEOUT_NS, 50_000_000)      # 50 ms
    ctx.set_option(m3d.OPT_TEST_WITHHOLD_TILE, 0)
    # the resident kernel streaming per-step operators (its tiles let their bulk copy in
    # flight land before they stop), interpolating in the kernel, and the persistent kernel
    for plan, stepop in ((m3d.PLAN_RESIDENT, 1), (m3d.PLAN_RESIDENT, 0), (m3d.PLAN_PERSISTENT, 0)):
        ctx.set_option(m3d.OPT_YEAR_PLAN, plan)
        ctx.set_option(m3d.OPT_STEP_OPERATORS, stepop)
        ctx.year_map(y0, y1, u)
        with pytest.raises(m3d.Metos3dError) as e:
            ctx.sync()
        assert e.value.status == m3d.M3D_ERR_TIMEOUT
    ctx.set_option(m3d.OPT_STEP_OPERATORS, 1)
    ctx.set_option(m3d.OPT_YEAR_PLAN, m3d.PLAN_RESIDENT)
    ctx.set_option(m3d.OPT_TEST_WITHHOLD_TILE, -1)
    ctx.set_option(m3d.OPT_WAIT_TIMEOUT_NS, 2_000_000_000)
    ctx.year_map(y0, y1, u)
    ctx.sync()
    assert rel_err(y1.cpu().numpy(), oracle.year_map(P, y0_h, u_h)) < YEAR_TOL
    ctx.close()


def test_year_map_in_place_and_repeatable(m3d):
    p, P = problem("tiny_6x4x4")
    u = mi.default_params_ndop()
    ctx = ctx_for(m3d, p)
    y0 = mi.random_state(p)
    a = cuda(y0)
    b = torch.empty_like(a)
    ctx.year_map(a, b, cuda(u))
    ctx.year_map(a, a, cuda(u))          # y0 and y1 may alias
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    ctx.close()


def test_year_map_host_matches_device(m3d):
    p, P = problem("tiny_6x4x4")
    u = mi.default_params_ndop()
    ctx = ctx_for(m3d, p)
    y0 = mi.random_state(p)
    got = ctx.year_map_host(y0, u)
    d = torch.empty((2, p.n), dtype=torch.float64, device="cuda")
    ctx.year_map(cuda(y0), d, cuda(u))
    torch.cuda.synchronize()
    assert np.array_equal(got, d.cpu().numpy())
    ctx.close()


def test_transport_only_year_map(m3d):
    p, P = problem("tiny_6x4x4")
    ctx = ctx_for(m3d, p, model=m3d.MODEL_NONE, ntracer=3, nparam=0)
    y0 = mi.random_state(p, ntracer=3)
    d = torch.empty((3, p.n), dtype=torch.float64, device="cuda")
    ctx.year_map(cuda(y0), d, None)
    torch.cuda.synchronize()
    assert rel_err(d.cpu().numpy(), oracle.year_map(P, y0, np.zeros(0), model=oracle.MODEL_NONE)) < YEAR_TOL
    ctx.close()


# ------------------------------------------------------------------ diagnostics and errors
def test_residual_and_mass(m3d):
    p, _ = problem("ndop_64x32x8")
    ctx = ctx_for(m3d, p)
    a = mi.random_state(p)
    b = mi.random_state(p, seed=99)
    assert abs(ctx.residual(cuda(a), cuda(b)) / np.linalg.norm(a - b) - 1) < 1e-13
    assert abs(ctx.mass(cuda(a)) / math.fsum((p.vol * a).ravel()) - 1) < 1e-13
    ctx.close()


def test_nonfinite_is_reported(m3d):
    p, _ = problem("tiny_4x3x3")
    ctx = ctx_for(m3d, p)
    y = mi.random_state(p)
    assert ctx.check_finite(cuda(y)) == m3d.M3D_OK
    y[1, 5] = np.nan
    assert ctx.check_finite(cuda(y)) == m3d.M3D_ERR_NONFINITE
    ctx.close()


def test_bad_arguments_are_rejected(m3d):
    p, _ = problem("tiny_4x3x3")
    with pytest.raises(m3d.Metos3dError) as e:
        m3d.Context.from_problem(p, model=m3d.MODEL_NDOP, ntracer=3, nparam=7)
    assert e.value.status == m3d.M3D_ERR_ARG
    bad = np.array(p.exp_colidx, copy=True)
    bad[3] = p.n + 5
    with pytest.raises(m3d.Metos3dError) as e:
        m3d.Context(col_start=p.col_start, h=p.h, zc=p.zc, vol=p.vol, lat=p.lat, exp_rowptr=p.exp_rowptr,
                    exp_colidx=bad, exp_val=p.exp_val, imp_blk=p.imp_blk)
    assert e.value.status == m3d.M3D_ERR_ARG
    ctx = ctx_for(m3d, p)
    y = cuda(mi.random_state(p))
    with pytest.raises(m3d.Metos3dError):
        ctx.step(2880, y, torch.empty_like(y), cuda(mi.default_params_ndop()))
    with pytest.raises(m3d.Metos3dError):
        ctx.step(0, y, y, cuda(mi.default_params_ndop()))       # in place is not allowed for one step
    ctx.close()
