"""Pins of the oracle's spin-up and Newton-Krylov solve (Sections 4, 6, 7).

Newton's method and the spin-up (plain fixed-point iteration of the year map) are different
algorithms for the same periodic solution; for a fixed total mass it is unique.  The
globalisation the paper names (Section 6: backtracking line search with cubic interpolation,
Eisenstat-Walker inner tolerances) is pinned piece by piece: the forcing terms against
values of the Eisenstat-Walker choice-2 rule evaluated in exact arithmetic, the backtracks
against minimisers of polynomial models fitted by an independent linear solve, the line
search's slope against a direct Jacobian product, and a far start on which the solver really
backtracks.  A mutation check plants mistakes in a copy of the solver and runs these pins.
"""
import importlib.util
import math
import os

import numpy as np
import pytest

import m3d_inputs as mi
import oracle
from oracle import newton as on

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Far start on which Newton backtracks (quadratic and cubic steps) and still converges:
# N x 10 of the constant initial state, alpha at 1.5 x its default (the top of the ensemble's
# range), tangent products.  Its path (iteration counts, steps tried) stays the same when the
# start is perturbed by 1e-12, so a solver that differs from this one by rounding (another
# compiler's libm, the GPU) takes the same path.
FAR_SCALE = (10.0, 1.0)
FAR_U = (1.0, 1.5, 1.0, 1.0, 1.0, 1.0, 1.0)


@pytest.fixture(scope="module")
def tiny():
    p = mi.make_problem("tiny_6x4x4")
    return p, oracle.Problem(p)


@pytest.fixture(scope="module")
def newton_solution(tiny):
    p, P = tiny
    y0 = mi.initial_state(p)
    y, rep = on.newton_krylov(P, y0, mi.default_params_ndop(), tol=1e-8)
    return y0, y, rep


def far_case(p):
    u = mi.default_params_ndop() * np.array(FAR_U)
    y0 = mi.initial_state(p) * np.array(FAR_SCALE)[:, None]
    return y0, u


@pytest.fixture(scope="module")
def far_solution(tiny):
    p, P = tiny
    y0, u = far_case(p)

    def tan(y, py, v):
        return oracle.year_tangent(P, y, v, u)[1]

    y, rep = on.newton_krylov(P, y0, u, tol=1e-8, jv=tan, record_steps=True)
    return y0, u, y, rep


# ---- the pieces, as functions of the module under test (the mutation check reuses them)

def hermite_fit(xs_vals, f0, slope):
    """Coefficients c[0..d] of the polynomial with p(0) = f0, p'(0) = slope and p(x) = v at the
    given (x, v) pairs, by solving the linear interpolation conditions."""
    d = 1 + len(xs_vals)
    A = np.zeros((d + 1, d + 1))
    rhs = np.zeros(d + 1)
    A[0, 0], rhs[0] = 1.0, f0
    A[1, 1], rhs[1] = 1.0, slope
    for row, (x, v) in enumerate(xs_vals, start=2):
        A[row] = [x ** k for k in range(d + 1)]
        rhs[row] = v
    return np.linalg.solve(A, rhs)


def poly_local_min(c, lo, hi):
    """The local minimiser of the polynomial with coefficients c (ascending) in (lo, hi)."""
    P = np.polynomial.Polynomial(c)
    cands = [x.real for x in P.deriv().roots() if abs(x.imag) < 1e-12 and lo < x.real < hi
             and P.deriv(2)(x.real) > 0]
    assert len(cands) == 1, cands
    return cands[0]


def pins_forcing_term(m):
    # exact values of the choice-2 rule (gamma = 0.9, alpha = the golden ratio), evaluated in
    # exact arithmetic
    assert m.forcing_term(5.0, None, None, 1e-8) == 0.3                       # first step
    # r/r_prev = 0.1, eta_prev = 0.2: safeguard 0.9 * 0.2^alpha = 0.0666 <= 0.1 not applied
    assert math.isclose(m.forcing_term(1.0, 10.0, 0.2, 1e-8), 0.021687451488674146, rel_tol=1e-13)
    # eta_prev = 0.8: safeguard 0.9 * 0.8^alpha = 0.6272 > 0.1 raises the 0.0217
    assert math.isclose(m.forcing_term(1.0, 10.0, 0.8, 1e-8), 0.62724732019365146, rel_tol=1e-13)
    # the safeguard threshold: eta_prev = (1/9)^(1/alpha) = 0.25719 gives exactly 0.1
    assert math.isclose(m.forcing_term(1.0, 10.0, 0.2572, 1e-8), 0.1000, rel_tol=1e-3)
    assert math.isclose(m.forcing_term(1.0, 10.0, 0.2571, 1e-8), 0.021687451488674146, rel_tol=1e-13)
    # the residual grew: 0.9 * 2^alpha = 2.76 is capped at 0.9
    assert m.forcing_term(2.0, 1.0, 0.3, 1e-8) == 0.9
    # near convergence: 0.9 * (1e-4)^alpha = 3.0e-7 is raised to 0.5 tol / r = 0.05
    assert math.isclose(m.forcing_term(1e-7, 1e-3, 0.01, 1e-8), 0.05, rel_tol=1e-13)


def pins_backtracks(m):
    # the quadratic model's minimiser: for an f that is a quadratic, the exact minimiser
    f0, slope, c = 2.0, -3.0, 5.0
    for lam in (1.0, 0.37):
        fl = f0 + slope * lam + c * lam * lam
        assert math.isclose(m.quadratic_backtrack(f0, slope, lam, fl), -slope / (2 * c), rel_tol=1e-13)
    # against the Hermite fit of arbitrary trial values
    for lam, fl in ((1.0, 2.5), (0.4, 1.9), (0.8, 7.0)):
        want = poly_local_min(hermite_fit([(lam, fl)], f0, slope), 0.0, 10.0)
        assert math.isclose(m.quadratic_backtrack(f0, slope, lam, fl), want, rel_tol=1e-12)
    # the cubic model's local minimiser for trials of a cubic and of other functions
    for (a, b) in ((0.7, 1.3), (-0.4, 2.0), (3.0, -0.5)):
        cubic = np.polynomial.Polynomial([f0, slope, b, a])
        for lam, lam_prev in ((0.3, 1.0), (0.05, 0.2)):
            got = m.cubic_backtrack(f0, slope, lam, cubic(lam), lam_prev, cubic(lam_prev))
            want = poly_local_min([f0, slope, b, a], 0.0, 50.0)
            assert math.isclose(got, want, rel_tol=1e-9), (a, b, lam, got, want)
    for lam, fl, lp, fp in ((0.3, 1.95, 1.0, 2.6), (0.1, 1.8, 0.45, 2.2), (0.2, 2.1, 0.5, 2.9)):
        c3 = hermite_fit([(lam, fl), (lp, fp)], f0, slope)
        want = poly_local_min(c3, 0.0, 50.0)
        assert math.isclose(m.cubic_backtrack(f0, slope, lam, fl, lp, fp), want, rel_tol=1e-9)
    # a cubic model with a = 0 is the quadratic
    quad = np.polynomial.Polynomial([f0, slope, 4.0])
    assert math.isclose(m.cubic_backtrack(f0, slope, 0.5, quad(0.5), 1.0, quad(1.0)), -slope / 8.0, rel_tol=1e-12)


def pins_line_search(m):
    """Newton on the scalar F(x) = atan(x) from x0 = 10: the full step overshoots to -138.6."""
    x0 = 10.0
    Fx = math.atan(x0)
    s = -Fx * (1.0 + x0 * x0)                       # the exact Newton step F / F'

    def f(lam):
        return 0.5 * math.atan(x0 + lam * s) ** 2

    f0 = f(0.0)
    slope = -2.0 * f0                               # F F' s = -F^2 for an exact Newton step
    lam, fl, trials = m.line_search(f, f0, slope)
    assert len(trials) >= 3 and trials[0][0] == 1.0
    for (l, v) in trials[:-1]:
        assert v > f0 + 1e-4 * l * slope            # every rejected trial fails the Armijo test
    assert fl <= f0 + 1e-4 * lam * slope and fl == f(lam) and (lam, fl) == trials[-1]
    for k in range(1, len(trials)):
        prev = trials[k - 1]
        if k == 1:
            model = hermite_fit([prev], f0, slope)
        else:
            model = hermite_fit([prev, trials[k - 2]], f0, slope)
        xm = poly_local_min(model, 0.0, 10.0)
        want = min(max(xm, 0.1 * prev[0]), 0.5 * prev[0])
        assert math.isclose(trials[k][0], want, rel_tol=1e-9), (k, trials, want)


def pins_line_search_bounds(m):
    """Quadratic f(lam) = f0 + slope lam + c lam^2, whose model minimiser -slope / (2c) the
    backtrack finds exactly: the Armijo test's side and the [0.1, 0.5] bounds on the next step."""
    f0, slope = 1.0, -2.0
    # f(1) lies between f0 + 1e-4 slope (the Armijo line) and f0 - 1e-4 slope: rejected; the
    # minimiser 0.500025 is capped at 0.5, where the decrease is ample
    c = -slope * (1.0 - 0.5e-4)
    lam, fl, trials = m.line_search(lambda x: f0 + slope * x + c * x * x, f0, slope)
    assert [t[0] for t in trials] == [1.0, 0.5]
    # a steep quadratic: the minimiser 0.005 is raised to 0.1 of the failed step
    c = -slope * 100.0
    lam, fl, trials = m.line_search(lambda x: f0 + slope * x + c * x * x, f0, slope)
    assert trials[1][0] == 0.1 and lam < 0.1


def pins_line_search_guards(m):
    """Trials outside the function's domain (not finite) and a search that finds no decrease."""
    f0, slope = 1.0, -2.0

    def f(x):                       # not defined beyond 0.5; below it f = 1 - 2x + 40x^2
        return math.nan if x > 0.5 else f0 + slope * x + 40.0 * x * x
    lam, fl, trials = m.line_search(f, f0, slope)
    # the NaN at 1 gives no model: the next trial is 0.1 of it; the failure there starts the
    # quadratic model afresh, whose minimiser 0.025 (in [0.01, 0.05]) is accepted
    assert [t[0] for t in trials][:2] == [1.0, 0.1] and math.isnan(trials[0][1]) and len(trials) == 3
    assert math.isclose(lam, 0.025, rel_tol=1e-12) and fl == f(lam)
    lam, fl, trials = m.line_search(lambda x: math.inf if x > 0.05 else f0 + slope * x, f0, slope)
    assert len(trials) == 3 and math.isclose(lam, 0.01, rel_tol=1e-12)
    # f increases along the direction: every step length down to 1e-4 fails, none below it is
    # tried, and the search returns no step
    lam, fl, trials = m.line_search(lambda x: f0 + x, f0, slope)
    assert lam == 0.0 and fl == f0 and 4 <= len(trials) <= 14
    assert min(t[0] for t in trials) >= 1e-4 and all(t[1] > f0 for t in trials)
    # the driver stops at its iterate when the line search fails: phi = 0 with a wrong
    # derivative (phi' = 2 I) makes the Newton step s = F an ascent direction of |F|
    y0 = np.array([1.0, -2.0, 0.5])
    y, rep = m.newton_solve(lambda y: np.zeros_like(y), y0, jv=lambda y, py, v: 2.0 * v)
    assert rep["line_search_failed"] and not rep["converged"] and np.array_equal(y, y0)
    assert rep["lambdas"] == [0.0] and rep["residuals"] == [float(np.linalg.norm(y0))] * 2
    # a start whose residual is not finite takes no step
    y, rep = m.newton_solve(lambda y: np.full_like(y, math.nan), y0)
    assert not rep["converged"] and rep["krylov"] == [] and np.array_equal(y, y0)


def pins_newton_driver(m):
    """The generic driver on F(y) = atan(A y - b) (componentwise, n = 6) from far away, where
    full Newton steps overshoot: exact Jacobian, every slope equal to F.J s computed directly,
    every GMRES step within its forcing term, quadratic and cubic backtracks on the way."""
    rng = np.random.default_rng(2)
    A = np.eye(6) + 0.3 * rng.standard_normal((6, 6)) / math.sqrt(6)
    bv = rng.standard_normal(6)

    def phi(y):
        return y - np.arctan(A @ y - bv)

    def jv(y, py, v):
        return v - (A @ v) / (1.0 + (A @ y - bv) ** 2)

    y0 = np.linalg.solve(A, bv + 8.0 * rng.standard_normal(6))
    y, rep = m.newton_solve(phi, y0, tol=1e-12, jv=jv, record_steps=True)
    assert rep["converged"] and np.linalg.norm(y - phi(y)) <= 1e-12
    assert np.linalg.norm(A @ y - bv) <= 1e-11                 # the root of F
    for k, (yk, sk) in enumerate(zip(rep["states"], rep["steps"])):
        Fk = yk - phi(yk)
        Js = sk - jv(yk, None, sk)
        assert math.isclose(rep["slopes"][k], float(Fk @ Js), rel_tol=1e-9, abs_tol=1e-14 * (Fk @ Fk))
        r = rep["residuals"][k]
        assert np.linalg.norm(Fk + Js) <= rep["etas"][k] * r * (1 + 1e-9)      # GMRES met eta
        if k > 0:
            assert rep["etas"][k] == pytest.approx(
                min(max(max(0.9 * (r / rep["residuals"][k - 1]) ** ((1 + math.sqrt(5)) / 2),
                            0.9 * rep["etas"][k - 1] ** ((1 + math.sqrt(5)) / 2)
                            if 0.9 * rep["etas"][k - 1] ** ((1 + math.sqrt(5)) / 2) > 0.1 else 0.0),
                        0.5e-12 / r), 0.9), rel=1e-12)
    assert any(len(t) == 2 for t in rep["trials"]) and any(len(t) >= 4 for t in rep["trials"])


def test_forcing_term_is_eisenstat_walker_choice_2():
    pins_forcing_term(on)


def test_backtracks_minimise_their_polynomial_models():
    pins_backtracks(on)


def test_line_search_on_a_scalar_newton_step():
    pins_line_search(on)


def test_line_search_bounds_and_armijo_side():
    pins_line_search_bounds(on)


def test_newton_driver_slopes_and_forcing_on_a_small_map():
    pins_newton_driver(on)


def test_line_search_outside_the_domain_and_when_it_finds_no_decrease():
    pins_line_search_guards(on)


def test_gmres_mgs_solves_a_small_system():
    r = np.random.default_rng(0)
    A = np.eye(30) + 0.3 * r.standard_normal((30, 30)) / math.sqrt(30)
    b = r.standard_normal(30)
    for restart in (30, 7):                  # full and restarted
        x, it, res = on.gmres_mgs(lambda v: A @ v, b, 1e-12, restart, 500)
        assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)


def test_gmres_slope_identity_with_the_tangent(tiny):
    """F.J s = -(|F|^2 - rho^2) for GMRES's step on the year map's Newton system, J s taken
    directly from the oracle's tangent year map."""
    p, P = tiny
    u = mi.default_params_ndop()
    y = mi.random_state(p, seed=4)
    py, _ = oracle.year_tangent(P, y, np.zeros_like(y), u)
    F = (y - py).ravel()

    def J(v):
        return v - oracle.year_tangent(P, y, v.reshape(y.shape), u)[1].ravel()

    for eta in (0.5, 0.05):
        s, its, res_rel = on.gmres_mgs(J, -F, eta, 200, 200)
        rho = res_rel * np.linalg.norm(F)
        assert rho <= eta * np.linalg.norm(F) * (1 + 1e-12) and its >= 1
        assert math.isclose(float(F @ J(s)), -(F @ F - rho * rho), rel_tol=1e-8)


def test_newton_converges_and_keeps_mass(tiny, newton_solution):
    p, P = tiny
    y0, y, rep = newton_solution
    assert rep["converged"] and rep["residuals"][-1] < 1e-8
    assert len(rep["residuals"]) <= 12
    # the residual really is ||phi(y) - y|| at the returned state
    py = oracle.year_map(P, y, mi.default_params_ndop())
    assert np.linalg.norm((py - y).ravel()) < 1e-8
    m0 = math.fsum((p.vol * y0).ravel())
    assert abs(math.fsum((p.vol * y).ravel()) / m0 - 1) < 1e-13


def test_newton_backtracks_from_a_far_start(tiny, far_solution):
    """Quadratic and cubic backtracks on the year map, then quadratic convergence."""
    p, P = tiny
    y0, u, y, rep = far_solution
    assert rep["converged"]
    assert np.linalg.norm((oracle.year_map(P, y, u) - y).ravel()) < 1e-8
    assert any(len(t) == 2 for t in rep["trials"]) and any(len(t) >= 3 for t in rep["trials"])
    assert min(rep["lambdas"]) < 0.5
    for k, (yk, sk) in enumerate(zip(rep["states"], rep["steps"])):
        if rep["residuals"][k] < 1e-5:
            break                # below this, F = y - phi(y) itself carries relative rounding of 1e-6 and more
        yk = yk.reshape(y0.shape)
        Fk = (yk - oracle.year_map(P, yk, u)).ravel()
        Js = sk - oracle.year_tangent(P, yk, sk.reshape(y0.shape), u)[1].ravel()
        # to 1e-4: the step was projected on the zero-mass directions after GMRES, which moves
        # J s by a rounding-sized multiple of J w
        assert math.isclose(rep["slopes"][k], float(Fk @ Js), rel_tol=1e-4), k
    m0 = math.fsum((p.vol * y0).ravel())
    assert abs(math.fsum((p.vol * y).ravel()) / m0 - 1) < 1e-12


@pytest.mark.slow
def test_newton_agrees_with_long_spinup(tiny, newton_solution):
    """The paper's comparison: spin-up (fixed-point iteration) and Newton reach the same periodic state."""
    p, P = tiny
    y0, y, _ = newton_solution
    ys, hist = on.spinup(P, y0, mi.default_params_ndop(), 1500)
    assert hist[-1] < 1e-11
    big = [h for h in hist if h > 1e-10]                # above the rounding floor the decay is monotone
    assert hist[0] > 1.0 and all(b < a * 1.0001 for a, b in zip(big[50:], big[51:]))
    assert np.abs(ys - y).max() / np.abs(y).max() < 1e-7


def test_tangent_product_option_matches_fd(tiny):
    """With an exact phi'(y) v (here: central differences of the oracle), Newton converges too."""
    p, P = tiny
    u = mi.default_params_ndop()

    def jv(y, py, v):
        h = 1e-6 * np.linalg.norm(y) / np.linalg.norm(v)
        return (oracle.year_map(P, y + h * v, u) - oracle.year_map(P, y - h * v, u)) / (2 * h)

    y, rep = on.newton_krylov(P, mi.initial_state(p), u, tol=1e-8, jv=jv)
    assert rep["converged"]


# ---- mutation check of the solver's pins: each mistake, planted in a copy of the solver,
# fails at least one of the pins above
NEWTON_MUTANTS = {
    "cubic_a_sign": ("a = (r1 / (lam * lam) - r2", "a = (r1 / (lam * lam) + r2"),
    "cubic_b_sign": ("b = (-lam_prev * r1", "b = (lam_prev * r1"),
    "cubic_root_branch": ("(-b + math.sqrt(disc))", "(-b - math.sqrt(disc))"),
    "quadratic_factor": ("(2.0 * (f_lam - f0 - slope * lam))", "(f_lam - f0 - slope * lam)"),
    "quadratic_lam_power": ("-slope * lam * lam /", "-slope * lam /"),
    "eta_exponent": ("eta = gamma * (r / r_prev) ** alpha", "eta = gamma * (r / r_prev) ** 2"),
    "eta_safeguard_dropped": ("if safe > 0.1:", "if False:"),
    "eta_safeguard_exponent": ("safe = gamma * eta_prev ** alpha", "safe = gamma * eta_prev"),
    "eta_lower_clamp_dropped": ("max(eta, 0.5 * tol / r)", "max(eta, 0.0)"),
    "eta_cap_dropped": ("return min(max(eta, 0.5 * tol / r), eta_max)", "return max(eta, 0.5 * tol / r)"),
    "step_floor_dropped": ("lam = min(max(lt, lo * lam), hi * lam)", "lam = min(lt, hi * lam)"),
    "step_cap_dropped": ("lam = min(max(lt, lo * lam), hi * lam)", "lam = max(lt, lo * lam)"),
    "armijo_sign": ("fl <= f0 + armijo * lam * slope", "fl <= f0 - armijo * lam * slope"),
    "slope_of_exact_newton": ("slope = -(r * r - rho * rho)", "slope = -r * r"),
    "models_swapped": ("if prev is None:\n            lt = quadratic", "if prev is not None:\n            lt = quadratic"),
    "nonfinite_kept_as_model": ("prev = None\n            lam = lo * lam", "prev = (lam, fl)\n            lam = lo * lam"),
    "nonfinite_not_caught": ("if not math.isfinite(fl):", "if False:"),
    "failure_takes_the_last_step": ("return 0.0, f0, trials", "return trials[-1][0], trials[-1][1], trials"),
    "failure_below_lam_min_tried": ("while lam >= lam_min:", "while lam >= 0.1 * lam_min:"),
    "failure_not_stopping": ("if lam == 0.0:", "if False:"),
}


def _mutant_module(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "newton.py")).read()
    if name is not None:
        old, new = NEWTON_MUTANTS[name]
        assert src.count(old) >= 1, "mutation site not found: %s" % name
        src = src.replace(old, new, 1)
    name = name or "unmutated"
    path = tmp_path / ("newton_%s.py" % name)
    path.write_text(src.replace("from . import MODEL_NDOP, year_map", "from oracle import MODEL_NDOP, year_map"))
    spec = importlib.util.spec_from_file_location("newton_mutant_" + name, str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_unmutated_copy_passes_the_newton_pins(tmp_path):
    """The control: the solver's own source, copied and loaded as the mutants are, passes
    every pin, so a mutant fails because of its mistake and not because of the copy."""
    mod = _mutant_module(None, tmp_path)
    for pins in (pins_forcing_term, pins_backtracks, pins_line_search, pins_line_search_bounds,
                 pins_line_search_guards, pins_newton_driver):
        pins(mod)


@pytest.mark.parametrize("name", sorted(NEWTON_MUTANTS))
def test_newton_pins_catch_mutant(name, tmp_path):
    mod = _mutant_module(name, tmp_path)
    caught = False
    for pins in (pins_forcing_term, pins_backtracks, pins_line_search, pins_line_search_bounds,
                 pins_line_search_guards, pins_newton_driver):
        try:
            pins(mod)
        except (AssertionError, ValueError, TypeError, ZeroDivisionError, KeyError, np.linalg.LinAlgError,
                RuntimeError):
            caught = True
            break
    assert caught, "the Newton pins did not catch mutant %s" % name
