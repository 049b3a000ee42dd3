"""The numbers the paper prints about its set-up, read from tests/golden/, against the
synthetic inputs, the oracle and the library's defaults (no GPU needed).

The paper's result figures carry no values; what it does print (Section 7) is the size of its
2.8125-degree grid, the length of a model year, the model configuration and the GMRES
restart.  The synthetic stand-in grid and the solvers' defaults must match them.
"""
import ctypes
import os

import numpy as np
import pytest

import m3d_inputs as mi

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_section7_setup.txt")


def _facts():
    facts = {}
    for line in open(GOLDEN):
        body = line.split("#", 1)[0].split()
        if body:
            key, value = body
            facts[key] = float(value) if "." in value else int(value)
    return facts


FACTS = _facts()


def test_fixture_is_complete_and_cited():
    assert set(FACTS) == {"grid_resolution_deg", "layers", "cells_per_tracer", "steps_per_year",
                          "monthly_matrices", "euphotic_layers", "internal_steps", "gmres_restart"}
    for line in open(GOLDEN):
        if line.split("#", 1)[0].strip():
            assert "# Section" in line, line


def test_stand_in_grid_has_the_papers_size():
    sp = mi.spec("ndop_128x64x15")
    p = mi.make_problem("ndop_128x64x15")
    assert 360.0 / sp.nx == FACTS["grid_resolution_deg"] and 180.0 / sp.ny == FACTS["grid_resolution_deg"]
    assert p.lmax == FACTS["layers"] and len(sp.h) == FACTS["layers"]
    assert p.n == FACTS["cells_per_tracer"]
    assert p.nstep == FACTS["steps_per_year"] and p.nmonth == FACTS["monthly_matrices"]
    assert p.exp_val.shape[0] == FACTS["monthly_matrices"] and p.imp_blk.shape[0] == FACTS["monthly_matrices"]


def test_source_term_acts_in_the_papers_euphotic_layers():
    """Uptake only in the top euphotic_layers layers: with no DOP and no light-independent
    term, the oracle's PO4-DOP increment takes PO4 there and returns it below."""
    import oracle
    L = 6
    h = np.array([50.0, 70.0, 90.0, 110.0, 130.0, 150.0])
    d = np.cumsum(h) - 0.5 * h
    y = np.stack([np.full(L, 2.17), np.zeros(L)])
    u = mi.default_params_ndop()
    dy = oracle.bgc(y, h, d, u, insol=400.0, model=mi.MODEL_NDOP)
    neu = FACTS["euphotic_layers"]
    assert np.all(dy[0, :neu] < 0.0) and np.all(dy[0, neu:] > 0.0)


def test_solvers_default_to_the_papers_restart():
    import inspect
    from oracle import newton as on
    assert inspect.signature(on.newton_krylov).parameters["restart"].default == FACTS["gmres_restart"]
    import paper_1410_0204_gb300 as m3d
    from paper_1410_0204_gb300 import binding as bd, build as b
    b.build()
    L = m3d.load()
    o = bd.NewtonOptions()
    L.metos3d_newton_default_options(ctypes.byref(o))
    assert o.restart == FACTS["gmres_restart"]


def test_model_interface_takes_the_papers_internal_steps():
    """Eight internal Euler steps of length dt/8 (the paper's runs) give the same increment as
    one step of dt/8 applied eight times in turn."""
    import oracle
    L = 4
    h = np.array([50.0, 70.0, 90.0, 110.0])
    d = np.cumsum(h) - 0.5 * h
    y = np.stack([np.full(L, 2.17), np.full(L, 0.3)])
    u = mi.default_params_ndop()
    nsub = FACTS["internal_steps"]
    dt = 1.0 / FACTS["steps_per_year"]
    whole = oracle.bgc(y, h, d, u, dt=dt, insol=400.0, model=mi.MODEL_NDOP, nsub=nsub)
    yk = y.copy()
    for _ in range(nsub):
        yk = yk + oracle.bgc(yk, h, d, u, dt=dt / nsub, insol=400.0, model=mi.MODEL_NDOP, nsub=1)
    np.testing.assert_allclose(whole, yk - y, rtol=1e-13, atol=1e-16)
