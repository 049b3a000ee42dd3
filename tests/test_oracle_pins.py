"""Pins of the CPU oracle against what the paper and the mathematics fix.

The paper prints no worked example and no result values (its figures are empty), so the
oracle is pinned by brute force on tiny grids, closed forms of special cases of the
PO4-DOP model (Section 2.2.1), textbook values of the insolation, and invariants of the
method (mass conservation, positivity, constant fields under pure transport).
"""
import math

import numpy as np
import pytest

import m3d_inputs as mi
import oracle

DT = 1.0 / 2880


@pytest.fixture(scope="module")
def tiny():
    p = mi.make_problem("tiny_4x3x3")
    return p, oracle.Problem(p)


@pytest.fixture(scope="module")
def tiny6():
    p = mi.make_problem("tiny_6x4x4")
    return p, oracle.Problem(p)


def _identity_transport(p):
    """A copy of p whose explicit and implicit matrices are the identity."""
    import copy
    q = copy.copy(p)
    rows = np.repeat(np.arange(p.n), np.diff(p.exp_rowptr))
    ev = np.where(rows == p.exp_colidx, 1.0, 0.0)
    q.exp_val = np.tile(ev, (p.nmonth, 1))
    ib = np.zeros(p.s_imp)
    for c in range(p.ncol):
        L = int(p.nlayer[c])
        ib[p.blk_off[c]:p.blk_off[c] + L * L] = np.eye(L).ravel()
    q.imp_blk = np.tile(ib, (p.nmonth, 1))
    return q


# ----------------------------------------------------------------------------- time weights
def test_month_weights_on_month_centres():
    # reading: monthly matrices sit at mid-month, so the operator at t = (m + 1/2)/12 is month m alone
    for m in range(12):
        m0, m1, w = oracle.month_weights(240 * m + 120)
        assert (m0, m1, w) == (m, (m + 1) % 12, 0.0)


def test_month_weights_at_month_boundaries_and_linear():
    m0, m1, w = oracle.month_weights(0)
    assert (m0, m1, w) == (11, 0, 0.5)           # Jan 1: halfway between December and January
    ws = [oracle.month_weights(j) for j in range(2880)]
    for j in range(2879):
        a, b = ws[j], ws[j + 1]
        if a[0] == b[0]:
            assert abs((b[2] - a[2]) - 1.0 / 240) < 1e-15
        else:
            assert b[0] == a[1] and abs(a[2] + 1.0 / 240 - 1.0) < 1e-12 and b[2] == 0.0
    assert all(0.0 <= w < 1.0 for _, _, w in ws)


# ----------------------------------------------------------------------------- brute force
def test_step_is_month_operator_at_month_centre(tiny):
    p, P = tiny
    y = mi.random_state(p)
    for m in (0, 5, 11):
        j = 240 * m + 120
        A, B = p.dense_exp(m), p.dense_imp(m)
        got = oracle.step(P, j, y, mi.default_params_ndop(), model=oracle.MODEL_NONE)
        want = (B @ (A @ y.T)).T
        assert np.abs(got - want).max() < 1e-14


def test_step_between_months_is_average(tiny):
    p, P = tiny
    y = mi.random_state(p)
    A = 0.5 * (p.dense_exp(11) + p.dense_exp(0))
    B = 0.5 * (p.dense_imp(11) + p.dense_imp(0))
    got = oracle.step(P, 0, y, mi.default_params_ndop(), model=oracle.MODEL_NONE)
    assert np.abs(got - (B @ (A @ y.T)).T).max() < 1e-14


def test_year_map_equals_dense_product_of_steps(tiny):
    p, P = tiny
    y0 = mi.random_state(p)
    Ad = [p.dense_exp(m) for m in range(12)]
    Bd = [p.dense_imp(m) for m in range(12)]
    Phi = np.eye(p.n)
    for j in range(2880):
        m0, m1, w = oracle.month_weights(j)
        Aj = (1 - w) * Ad[m0] + w * Ad[m1]
        Bj = (1 - w) * Bd[m0] + w * Bd[m1]
        Phi = Bj @ (Aj @ Phi)
    got = oracle.year_map(P, y0, mi.default_params_ndop(), model=oracle.MODEL_NONE)
    want = (Phi @ y0.T).T
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-13


def test_equal_months_give_matrix_power(tiny6):
    import copy
    p0, _ = tiny6
    p = copy.copy(p0)
    p.exp_val = np.tile(p0.exp_val[3], (12, 1))
    p.imp_blk = np.tile(p0.imp_blk[7], (12, 1))
    P = oracle.Problem(p)
    y0 = mi.random_state(p)
    M = np.linalg.matrix_power(p.dense_imp(0) @ p.dense_exp(0), 2880)
    got = oracle.year_map(P, y0, mi.default_params_ndop(), model=oracle.MODEL_NONE)
    assert np.abs(got - (M @ y0.T).T).max() / np.abs(y0).max() < 1e-12


def test_constant_field_preserved_by_transport(tiny6):
    p, P = tiny6
    y0 = np.full((2, p.n), 1.75)
    got = oracle.year_map(P, y0, mi.default_params_ndop(), model=oracle.MODEL_NONE)
    assert np.abs(got - 1.75).max() < 1e-12


def test_step_composition_q_on_old_state(tiny6):
    """y_{j+1} = A_imp (A_exp y_j + bgc(y_j)): q acts on y_j, before the implicit part."""
    p, P = tiny6
    u = mi.default_params_ndop()
    y = mi.random_state(p)
    for j in (7, 1000, 2879):
        m0, m1, w = oracle.month_weights(j)
        A = (1 - w) * p.dense_exp(m0) + w * p.dense_exp(m1)
        B = (1 - w) * p.dense_imp(m0) + w * p.dense_imp(m1)
        z = (A @ y.T).T
        t = j / 2880
        for c in range(p.ncol):
            s, e = p.col_start[c], p.col_start[c + 1]
            insol, df = oracle.insolation(p.lat[c], t)
            z[:, s:e] += oracle.bgc(y[:, s:e], p.h[s:e], p.zc[s:e], u, t=t, insol=insol, dayfrac=df)
        want = (B @ z.T).T
        got = oracle.step(P, j, y, u)
        assert np.abs(got - want).max() < 1e-14


# ----------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("name", ["tiny_6x4x4", "ndop_64x32x8"])
def test_mass_conserved_over_a_year(name):
    p = mi.make_problem(name)
    P = oracle.Problem(p)
    y0 = mi.initial_state(p)
    u = mi.default_params_ndop()
    for nsub in (1, 8) if name.startswith("tiny") else (1,):
        y1 = oracle.year_map(P, y0, u, nsub=nsub)
        m0 = math.fsum((p.vol * y0).ravel())
        m1 = math.fsum((p.vol * y1).ravel())
        assert abs(m1 - m0) / m0 < 1e-12
        assert y1.min() > 0.0                                     # positivity


def test_nsub_changes_result_but_both_conserve(tiny6):
    p, P = tiny6
    y0 = mi.initial_state(p)
    u = mi.default_params_ndop()
    a = oracle.steps(P, 0, 240, y0, u, nsub=1)
    b = oracle.steps(P, 0, 240, y0, u, nsub=8)
    assert np.abs(a - b).max() > 1e-6
    for y in (a, b):
        assert abs(math.fsum((p.vol * y).ravel()) / math.fsum((p.vol * y0).ravel()) - 1) < 1e-13


# ----------------------------------------------------------------------------- closed forms of q
def test_dop_decay_closed_form(tiny6):
    """alpha = 0: no production, DOP_n = DOP_0 (1 - lambda dt/nsub)^(n nsub), N gains the rest."""
    p, _ = tiny6
    P = oracle.Problem(_identity_transport(p))
    u = mi.default_params_ndop()
    u[1] = 0.0
    y0 = mi.random_state(p)
    for nsub in (1, 8):
        y1 = oracle.year_map(P, y0, u, nsub=nsub)
        decay = (1.0 - u[3] * DT / nsub) ** (2880 * nsub)
        # rounding bound: one rounding per Euler substep, n = 2880 nsub of them
        tol = 4 * 2880 * nsub * np.finfo(float).eps
        assert np.abs(y1[1] / (y0[1] * decay) - 1).max() < tol
        assert np.abs(y1[0] / (y0[0] + y0[1] * (1 - decay)) - 1).max() < tol
    # and the closed form of the continuous decay is approached: exp(-lambda) after one year
    assert abs((1.0 - u[3] * DT / 8) ** (2880 * 8) - math.exp(-u[3])) < 1e-5


def _column(nl=8):
    h = np.array([50.0, 70.0, 100.0, 140.0, 190.0, 240.0, 290.0, 340.0][:nl])
    zt = np.concatenate([[0.0], np.cumsum(h)[:-1]])
    return h, zt + 0.5 * h, zt, zt + h


def test_martin_flux_power_law():
    """lambda = 0: the flux through each interface z >= z_eu is E (z/z_eu)^-b (Martin et al.)."""
    h, d, ztop, zbot = _column(8)
    u = mi.default_params_ndop()
    u[3] = 0.0
    u[2] = 0.3
    y = np.vstack([np.linspace(1.0, 2.0, 8), np.full(8, 0.1)])
    yb = oracle.bgc(y, h, d, u, insol=300.0)
    uptake = -np.sum(h[:2] * yb[0, :2])                 # = dt sum f_k h_k
    assert uptake > 0
    assert abs(np.sum(h[:2] * yb[1, :2]) - u[2] * uptake) < 1e-13       # sigma to DOP
    E = (1 - u[2]) * uptake
    zeu = zbot[1]
    # ybgc is y^(nsub) - y^(0): each entry carries a rounding of about eps |y|
    tol = 8 * np.finfo(float).eps * np.sum(h * np.abs(y).sum(0))
    for k in range(2, 8):                              # flux through the top interface of layer k
        below = np.sum(h[k:] * yb[0, k:])
        assert abs(below - E * (ztop[k] / zeu) ** (-u[6])) < tol
    assert np.all(yb[0, 2:] >= 0)                      # remineralisation is a source
    assert np.all(yb[1, 2:] == 0)


def test_michaelis_menten_half_saturation():
    h, d, _, _ = _column(4)
    u = mi.default_params_ndop()
    u[0] = 0.0          # no attenuation: I = 0.4 insol
    u[3] = 0.0
    y = np.vstack([np.full(4, u[4]), np.zeros(4)])     # N = K_N
    insol = u[5] / 0.4                                 # I = K_I
    yb = oracle.bgc(y, h, d, u, insol=insol)
    f = u[1] * 360.0 * 0.5 * 0.5
    assert abs(yb[0, 0] + DT * f) < 1e-15
    assert abs(yb[1, 0] - DT * u[2] * f) < 1e-15
    # saturation: f -> alpha
    y2 = np.vstack([np.full(4, 1e14), np.zeros(4)])
    yb2 = oracle.bgc(y2, h, d, u, insol=1e16)
    assert abs(yb2[0, 0] / (-DT * u[1] * 360.0) - 1) < 1e-12


def test_light_attenuation_e_folding():
    h, d, _, _ = _column(4)
    u = mi.default_params_ndop()
    u[0] = 1.0 / (d[1] - d[0])     # one e-folding between the two euphotic layer centres
    u[3] = 0.0
    u[5] = 1e12                    # K_I >> I: production linear in light
    y = np.vstack([np.full(4, 1.3), np.zeros(4)])
    yb = oracle.bgc(y, h, d, u, insol=200.0)
    # DOP starts at 0, so its increment dt sigma f_k carries no cancellation
    assert abs(yb[1, 1] / yb[1, 0] - math.exp(-1.0)) < 1e-9


@pytest.mark.parametrize("nl", [1, 2, 3, 8])
def test_column_conservation_random(nl):
    r = np.random.default_rng(7 + nl)
    h, d, _, _ = _column(8)
    h, d = h[:nl], d[:nl]
    for _ in range(20):
        u = mi.default_params_ndop() * r.uniform(0.5, 1.5, 7)
        y = r.uniform(0.0, 3.0, (2, nl))
        for nsub in (1, 8):
            yb = oracle.bgc(y, h, d, u, insol=r.uniform(0, 500), nsub=nsub)
            tot = np.sum(h * (yb[0] + yb[1]))
            # each increment y^(nsub) - y^(0) carries a rounding of about eps |y| per substep
            assert abs(tot) < 8 * nsub * np.finfo(float).eps * np.sum(h * np.abs(y).sum(0))


def test_euphotic_zone_is_two_layers():
    h, d, _, _ = _column(6)
    u = mi.default_params_ndop()
    u[3] = 0.0
    y = np.vstack([np.full(6, 2.0), np.zeros(6)])
    yb = oracle.bgc(y, h, d, u, insol=300.0)
    assert np.all(yb[0, :2] < 0) and np.all(yb[0, 2:] > 0)


# ----------------------------------------------------------------------------- insolation
def test_insolation_textbook_values():
    S0 = 1361.0
    t_equinox = 0.25 - 10.0 / 360       # declination zero (March equinox)
    q, df = oracle.insolation(0.0, t_equinox)
    assert abs(q - S0 / math.pi) < 1e-9 and abs(df - 0.5) < 1e-15
    t_dec = 1.0 - 10.0 / 360            # December solstice: declination -23.44 degrees
    q, df = oracle.insolation(80.0, t_dec)
    assert q == 0.0 and df == 0.0       # polar night
    t_jun = 0.5 - 10.0 / 360            # June solstice
    q, df = oracle.insolation(89.999999, t_jun)
    assert abs(q - S0 * math.sin(math.radians(23.44))) < 1e-3 and df == 1.0   # polar day
    for lat in (-60.0, -13.0, 0.0, 37.0, 71.0):
        for t in (0.03, 0.4, 0.77):
            a, _ = oracle.insolation(lat, t)
            b, _ = oracle.insolation(-lat, t + 0.5)
            assert abs(a - b) < 1e-9 * S0    # hemispheric symmetry half a year apart
            assert 0.0 <= a <= S0
