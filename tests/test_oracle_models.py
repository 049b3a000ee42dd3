"""Pins of the oracle's N, PO4-DOP-PHY and NPZD-DOP models.

The N model is the PO4-DOP model without DOP, PO4-DOP-PHY is the paper's second example
(Section 2.2.2), and NPZD-DOP extends it by zooplankton and sinking detritus.  Each is
pinned by reductions to a model pinned elsewhere (PO4-DOP, whose own pins are closed
forms), by conservation of phosphorus per cell and per column, by closed forms of special
cases (Holling saturation, upwind sinking) and by mass conservation of whole steps.
"""
import numpy as np
import pytest

import m3d_inputs as mi
import oracle

DT = 1.0 / 2880
INSOL = 300.0


def _column(nl, seed=0):
    r = np.random.default_rng(seed)
    h = 40.0 + 60.0 * r.random(nl)
    d = np.cumsum(h) - 0.5 * h
    return h, d


def _state(ntr, nl, seed=1, lo=0.02, hi=2.0):
    r = np.random.default_rng(seed)
    return lo + (hi - lo) * r.random((ntr, nl))


def _q(model, y, h, d, u, insol=INSOL):
    """q itself: the one-substep increment divided by dt."""
    return oracle.bgc(y, h, d, u, dt=DT, insol=insol, model=model) / DT


def _rand_params(model, seed):
    r = np.random.default_rng(seed)
    u = mi.default_params(model) * (0.5 + r.random(len(mi.MODELS[model].params)))
    for i, name in enumerate(mi.MODELS[model].params):
        if name in mi.MODELS[model].fractions:
            u[i] = min(u[i], 1.0)
    return u


# ----------------------------------------------------------------------------- conservation
@pytest.mark.parametrize("model", [mi.MODEL_N, mi.MODEL_PHY, mi.MODEL_NPZD])
@pytest.mark.parametrize("nl", [1, 2, 3, 9, 15])
def test_column_phosphorus_conserved(model, nl):
    # every model only moves phosphorus between tracers and layers: sum_k h_k sum_tr q = 0
    ntr = len(mi.MODELS[model].tracers)
    for seed in range(4):
        h, d = _column(nl, seed)
        y = _state(ntr, nl, seed + 10)
        u = _rand_params(model, seed + 20)
        q = _q(model, y, h, d, u)
        scale = np.abs(q).sum(axis=0) @ h
        assert abs(float((q.sum(axis=0) * h).sum())) <= 1e-13 * max(scale, 1.0)


def test_phy_losses_stay_in_the_cell():
    # without growth (mu_1 = 0) there is no export, so phosphorus is conserved cell by cell
    nl = 6
    h, d = _column(nl)
    y = _state(3, nl, 3)
    u = mi.default_params(mi.MODEL_PHY)
    u[0] = 0.0
    q = _q(mi.MODEL_PHY, y, h, d, u)
    np.testing.assert_allclose(q.sum(axis=0), 0.0, atol=1e-13 * np.abs(q).max())
    assert np.all(q[2] < 0)                                 # PHY decays (into DOP) ...
    np.testing.assert_allclose(q[0], 360.0 * u[4] * y[1], rtol=1e-10)   # ... PO4 gains remineralised DOP


def test_npzd_cellwise_conservation_without_sinking():
    nl = 7
    h, d = _column(nl)
    y = _state(5, nl, 4, lo=0.01, hi=1.0)
    u = _rand_params(mi.MODEL_NPZD, 5)
    u[12] = 0.0                                            # w_D
    q = _q(mi.MODEL_NPZD, y, h, d, u)
    np.testing.assert_allclose(q.sum(axis=0), 0.0, atol=1e-13 * np.abs(q).max())


# ----------------------------------------------------------------------------- reductions
@pytest.mark.parametrize("nl", [1, 2, 5, 15])
def test_n_model_is_po4_dop_without_dop(nl):
    # N model == PO4-DOP with sigma = 0 (all production exported), lambda = 0 and DOP = 0
    h, d = _column(nl, 7)
    N = _state(1, nl, 8)
    kw, alpha, KN, KI, b = 0.03, 0.7, 0.4, 25.0, 0.9
    qn = _q(mi.MODEL_N, N, h, d, np.array([kw, alpha, KN, KI, b]))
    y2 = np.vstack([N, np.zeros((1, nl))])
    q2 = _q(mi.MODEL_NDOP, y2, h, d, np.array([kw, alpha, 0.0, 0.0, KN, KI, b]))
    np.testing.assert_allclose(qn[0], q2[0], rtol=1e-13, atol=1e-13 * np.abs(q2[0]).max())
    assert np.all(q2[1] == 0.0)


@pytest.mark.parametrize("nl", [1, 2, 4, 12])
def test_phy_reduces_to_po4_dop(nl):
    # sigma_3 = 1 and no PHY losses keep PHY = c constant; then f_1 = mu_1 c N/(N+K_1) I/(I+K_I)
    # is the PO4-DOP production with alpha = mu_1 c, and q1, q2 are the PO4-DOP terms
    h, d = _column(nl, 11)
    c = 0.37
    y = _state(3, nl, 12)
    y[2] = c
    mu1, kw, K1, KI, l2, s2, b = 1.3, 0.025, 0.6, 35.0, 0.004, 0.6, 0.8
    u_phy = np.array([mu1, kw, K1, KI, l2, s2, 0.0, 0.0, 0.0, 1.0, b])
    q3 = _q(mi.MODEL_PHY, y, h, d, u_phy)
    u_ndop = np.array([kw, mu1 * c, s2, 360.0 * l2, K1, KI, b])   # lambda per year
    q2 = _q(mi.MODEL_NDOP, y[:2], h, d, u_ndop)
    for i in range(2):
        np.testing.assert_allclose(q3[i], q2[i], rtol=1e-12, atol=1e-12 * np.abs(q2).max())
    assert np.all(q3[2] == 0.0)


@pytest.mark.parametrize("nl", [1, 2, 6, 15])
def test_npzd_reduces_to_phy(nl):
    # no zooplankton and no detritus, no P mortality, no sinking: NPZD-DOP (N, P, 0, 0, DOP)
    # is PO4-DOP-PHY (N, DOP, P) with sigma_3 = 0 (no grazed fraction, hence no export)
    # and no PHY losses, mu_1 = mu_P, lambda'_2 = lambda_DOP
    h, d = _column(nl, 13)
    s = _state(3, nl, 14)
    N, P, DOP = s[0], s[1], s[2]
    kw, muP, KN, KI, lO = 0.015, 0.9, 0.45, 28.0, 0.02
    u_npzd = np.array([kw, muP, KN, KI, 1.1, 0.12, 0.7, 0.0, 0.8, 0.04, 0.0, lO, 0.0])
    y5 = np.vstack([N, P, np.zeros(nl), np.zeros(nl), DOP])
    q5 = _q(mi.MODEL_NPZD, y5, h, d, u_npzd)
    u_phy = np.array([muP, kw, KN, KI, lO, 0.5, 0.0, 0.0, 0.0, 0.0, 0.9])
    q3 = _q(mi.MODEL_PHY, np.vstack([N, DOP, P]), h, d, u_phy)
    tol = dict(rtol=1e-12, atol=1e-12 * np.abs(q3).max())
    np.testing.assert_allclose(q5[0], q3[0], **tol)
    np.testing.assert_allclose(q5[1], q3[2], **tol)
    np.testing.assert_allclose(q5[4], q3[1], **tol)
    assert np.all(q5[2] == 0.0) and np.all(q5[3] == 0.0)


# ----------------------------------------------------------------------------- closed forms
def _npzd_only(**kw):
    names = mi.MODELS[mi.MODEL_NPZD].params
    u = np.zeros(len(names))
    u[names.index("K_N")] = 0.5
    u[names.index("K_I")] = 30.0
    u[names.index("K_P")] = 0.1
    for k, v in kw.items():
        u[names.index(k)] = v
    return u


def test_holling_half_saturation_and_saturation():
    # with only grazing on (epsilon = 1), Z gains and P loses mu_Z Z P/(K_P + P):
    # half the maximum at P = K_P, the maximum mu_Z Z as P grows without bound
    nl = 4
    h, d = _column(nl)
    muZ, KP, Z = 0.8, 0.1, 0.3
    u = _npzd_only(mu_Z=muZ, epsilon=1.0)
    for P, frac in ((KP, 0.5), (1e4 * KP, 1e4 / (1e4 + 1.0))):
        y = np.vstack([np.full(nl, 1.0), np.full(nl, P), np.full(nl, Z), np.zeros(nl), np.zeros(nl)])
        q = _q(mi.MODEL_NPZD, y, h, d, u)
        np.testing.assert_allclose(q[2], frac * 360.0 * muZ * Z, rtol=1e-9)
        np.testing.assert_allclose(q[1], -frac * 360.0 * muZ * Z, rtol=1e-9)


def test_detritus_sinking_upwind_closed_form():
    # uniform detritus in equal layers: only the top layer loses (w D / h) and only the
    # bottom layer gains it; interior layers see equal in- and outflow
    nl = 5
    h = np.full(nl, 50.0)
    d = np.cumsum(h) - 0.5 * h
    wD, D0 = 2.0, 0.4
    u = _npzd_only(w_D=wD)
    y = np.vstack([np.zeros(nl), np.zeros(nl), np.zeros(nl), np.full(nl, D0), np.zeros(nl)])
    q = _q(mi.MODEL_NPZD, y, h, d, u)
    rate = 360.0 * wD * D0 / 50.0
    np.testing.assert_allclose(q[3], [-rate, 0.0, 0.0, 0.0, rate], atol=1e-12 * rate)


def test_phy_growth_half_saturation():
    # at N = K_1 and I = K_I the PO4 uptake is a quarter of mu_1 PHY; DOP gets sigma_2 sigma_3
    # of it, PHY keeps (1 - sigma_3), the rest is exported below the euphotic zone
    nl = 3
    h, d = _column(nl)
    kw, K1, KI, mu1, s2, s3, PHY = 0.02, 0.5, 30.0, 1.5, 0.6, 0.7, 0.2
    insol = KI / (0.4 * np.exp(-kw * d[0]))                 # I = K_I in the top layer
    y = np.vstack([np.full(nl, K1), np.zeros(nl), np.full(nl, PHY)])
    u = np.array([mu1, kw, K1, KI, 0.0, s2, 0.0, 0.0, 0.0, s3, 0.858])
    q = _q(mi.MODEL_PHY, y, h, d, u, insol=insol)
    f1 = 360.0 * mu1 * PHY * 0.25
    np.testing.assert_allclose(q[0, 0], -f1, rtol=1e-12)
    np.testing.assert_allclose(q[1, 0], s2 * s3 * f1, rtol=1e-12)
    np.testing.assert_allclose(q[2, 0], (1.0 - s3) * f1, rtol=1e-12)


# ----------------------------------------------------------------------------- whole steps
@pytest.mark.parametrize("model", [mi.MODEL_N, mi.MODEL_PHY, mi.MODEL_NPZD])
def test_steps_conserve_total_mass(model):
    p = mi.make_problem("tiny_6x4x4")
    P = oracle.Problem(p)
    ntr = len(mi.MODELS[model].tracers)
    y0 = mi.random_state(p, ntr, seed=3, scale=(2.0, 0.2, 0.1, 0.1, 0.05))
    u = mi.default_params(model)
    y1 = oracle.steps(P, 100, 60, y0, u, model=model)
    m0 = float((y0.sum(axis=0) * p.vol).sum())
    m1 = float((y1.sum(axis=0) * p.vol).sum())
    assert abs(m1 - m0) <= 1e-13 * m0
    assert np.all(np.isfinite(y1)) and np.all(y1 > 0)


def test_ensemble_members_are_independent():
    # the ensemble year map is each member's own year map, whatever the other members are
    p = mi.make_problem("tiny_4x3x3")
    P = oracle.Problem(p)
    ens = mi.make_ensemble(((mi.MODEL_N, 1), (mi.MODEL_NDOP, 1), (mi.MODEL_NPZD, 1)), seed=5)
    ys = [mi.initial_state(p, m.ntracer, mi.model_initial_values(m.model)) for m in ens]
    out = oracle.ensemble_steps(P, 0, 30, ys, ens)
    alone = oracle.steps(P, 0, 30, ys[1], ens[1].u, model=ens[1].model)
    assert np.array_equal(out[1], alone)
    assert [o.shape[0] for o in out] == [1, 2, 5]


def test_ensemble_draw_within_spread():
    ens = mi.make_ensemble()
    assert [m.model for m in ens] == [mi.MODEL_N] * 16 + [mi.MODEL_NDOP] * 32 + [mi.MODEL_NPZD] * 16
    assert sum(m.ntracer for m in ens) == 160
    for m in ens:
        base = mi.default_params(m.model)
        assert np.all(m.u >= 0.5 * base - 1e-15) and np.all(m.u <= 1.5 * base + 1e-15)
