"""Degenerate problems through the C ABI, single context (every plan) and ensemble, against the
oracle: one water column, one-layer columns only, a single monthly matrix, and a year of an odd
number of steps (the result then ends in the other half of the ping-pong buffers).

The problems are restrictions of the seeded tiny grids: a subset of the cells, the explicit
rows and entries among them, and the top-left part of each implicit block (still the inverse
of a tridiagonal matrix when whole columns, or only their top layers, are kept).  The years
keep the method's step length (2880 steps, or 2879 for the odd year): the explicit Euler
source terms are stable there, whereas with far fewer steps a year of the growth terms
amplifies rounding differences without bound and no parity check is meaningful.
"""
import copy
import os

import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from tests._util import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PLANS = {"resident": 2, "persistent": 0, "graph": 1}
YEAR_TOL = 1e-10


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    return m


def restrict(p, cols, top_layers=None, nmonth=None, nstep=None):
    """The problem on columns `cols` (their top `top_layers` layers), months [0, nmonth), nstep."""
    q = copy.copy(p)
    keep, col_start = [], [0]
    for c in cols:
        L = int(p.col_start[c + 1] - p.col_start[c])
        Lk = L if top_layers is None else min(L, top_layers)
        keep.extend(range(int(p.col_start[c]), int(p.col_start[c]) + Lk))
        col_start.append(col_start[-1] + Lk)
    keep = np.array(keep)
    new_index = -np.ones(p.n, dtype=np.int64)
    new_index[keep] = np.arange(keep.size)
    nm = p.nmonth if nmonth is None else nmonth
    rowptr, colidx, ents = [0], [], []
    for r in keep:
        for e in range(p.exp_rowptr[r], p.exp_rowptr[r + 1]):
            if new_index[p.exp_colidx[e]] >= 0:
                colidx.append(new_index[p.exp_colidx[e]])
                ents.append(e)
        rowptr.append(len(colidx))
    blocks, blk_off = [], [0]
    for c, cnew in zip(cols, range(len(cols))):
        L = int(p.col_start[c + 1] - p.col_start[c])
        Lk = col_start[cnew + 1] - col_start[cnew]
        B = p.imp_blk[:nm, p.blk_off[c]:p.blk_off[c] + L * L].reshape(nm, L, L)[:, :Lk, :Lk]
        blocks.append(B.reshape(nm, Lk * Lk))
        blk_off.append(blk_off[-1] + Lk * Lk)
    q.col_start = np.array(col_start, dtype=np.int32)
    for name in ("col_i", "col_j", "lat", "area"):
        setattr(q, name, np.asarray(getattr(p, name))[list(cols)])
    for name in ("layer", "h", "zc", "vol"):
        setattr(q, name, np.asarray(getattr(p, name))[keep])
    q.exp_rowptr = np.array(rowptr, dtype=np.int32)
    q.exp_colidx = np.array(colidx, dtype=np.int32)
    q.exp_val = np.ascontiguousarray(p.exp_val[:nm][:, ents])
    q.blk_off = np.array(blk_off, dtype=np.int64)
    q.imp_blk = np.ascontiguousarray(np.hstack(blocks))
    q.nmonth = nm
    if nstep is not None:
        q.nstep = nstep
        q.dt = 1.0 / nstep
    return q


def single_context_all_plans(m3d, q, y0, u):
    ctx = m3d.Context.from_problem(q, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    out = {}
    for plan, code in PLANS.items():
        ctx.set_option(m3d.OPT_YEAR_PLAN, code)
        if ctx.get_option(m3d.OPT_YEAR_PLAN) != code:
            continue                                   # a plan this problem cannot use
        y1 = torch.empty((2, q.n), dtype=torch.float64, device="cuda")
        ctx.year_map(torch.from_numpy(y0).cuda(), y1, torch.from_numpy(u).cuda())
        out[plan] = y1.cpu().numpy()
    ctx.close()
    return out


def ensemble_year(m3d, q, members, ys):
    ens = m3d.Ensemble.from_problem(q, members)
    Y = torch.from_numpy(np.vstack(ys)).cuda()
    Y1 = ens.year_map(Y, torch.empty_like(Y)).cpu().numpy()
    offs = ens.offsets
    ens.close()
    return [Y1[offs[m]:offs[m + 1]] for m in range(len(members))]


EVERY_MODEL = ((mi.MODEL_N, 1), (mi.MODEL_NDOP, 1), (mi.MODEL_PHY, 1), (mi.MODEL_NPZD, 1))


def check(m3d, q):
    P = oracle.Problem(q)
    u = mi.default_params_ndop()
    y0 = mi.random_state(q, seed=5)
    want = oracle.year_map(P, y0, u)
    got = single_context_all_plans(m3d, q, y0, u)
    assert "resident" in got or "persistent" in got or "graph" in got
    for plan, g in got.items():
        assert rel_err(g, want) <= YEAR_TOL, plan
    members = mi.make_ensemble(EVERY_MODEL, seed=9)
    ys = [mi.initial_state(q, m.ntracer, mi.model_initial_values(m.model)) for m in members]
    for m, (g, y, mem) in enumerate(zip(ensemble_year(m3d, q, members, ys), ys, members)):
        assert rel_err(g, oracle.year_map(P, y, mem.u, model=mem.model)) <= YEAR_TOL, m


def test_single_water_column(m3d):
    p = mi.make_problem("tiny_6x4x4")
    deepest = int(np.argmax(np.diff(p.col_start)))
    check(m3d, restrict(p, [deepest]))


def test_one_layer_columns_only(m3d):
    p = mi.make_problem("tiny_6x4x4")
    check(m3d, restrict(p, list(range(p.ncol)), top_layers=1))


def test_two_layer_columns_only(m3d):
    # every column is all euphotic: the export stays in the bottom layer
    p = mi.make_problem("tiny_6x4x4")
    check(m3d, restrict(p, list(range(p.ncol)), top_layers=2))


def test_one_month_and_an_odd_year(m3d):
    p = mi.make_problem("tiny_6x4x4")
    check(m3d, restrict(p, list(range(p.ncol)), nmonth=1, nstep=2879))
