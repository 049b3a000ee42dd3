"""The oracle's derivative pins catch plausible mistakes.

The tangent and the reverse (adjoint) of every model, of the internal Euler steps and of the
transport are written by hand in the oracle's C source, and the pins of
test_oracle_tangent.py, test_oracle_adjoint.py and test_oracle_model_derivatives.py check
them against central differences of the pinned forward models and against each other (the
dot-product identity).  Each case here plants one mistake in a copy of that source (on the
CPU only), in the derivative code alone -- the forward model stays correct, so the mistake
is one that a forward-only check cannot see -- builds it, and runs those pins against it:
they must fail for every mutant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tmm_oracle.c")
PINS = ["test_oracle_tangent.py", "test_oracle_adjoint.py", "test_oracle_model_derivatives.py"]

# name: (text in the derivative code, its replacement, which occurrence (0 = first))
MUTANTS = {
    # tangent of the PO4-DOP term (Section 2.2.1)
    "ndop_tangent_uptake_derivative": ("* (KN / ((N[k] + KN) * (N[k] + KN))) * LF * dN[k];",
                                       "* (KN / (N[k] + KN)) * LF * dN[k];", 0),
    "ndop_tangent_dop_sign": ("dqD[k] = sigma * df - lambda * dDOP[k];",
                              "dqD[k] = sigma * df + lambda * dDOP[k];", 0),
    "ndop_tangent_export_thickness": ("dE += (1.0 - sigma) * df * h[k];", "dE += (1.0 - sigma) * df;", 0),
    "ndop_tangent_aphotic_remin_dropped": ("dqN[k] = (dE * pt - dE * pb) / h[k] + lambda * dDOP[k];",
                                           "dqN[k] = (dE * pt - dE * pb) / h[k];", 0),
    "ndop_tangent_shallow_deposit_dropped": ("dqN[nlayer - 1] += dE / h[nlayer - 1];",
                                             "dqN[nlayer - 1] += 0.0 * dE;", 0),
    # tangents of the N, PO4-DOP-PHY and NPZD-DOP terms
    "n_tangent_martin_bottom": ("dq[k] = dE * (top - bot) / h[k];", "dq[k] = dE * top / h[k];", 0),
    "phy_tangent_quadratic_loss": ("double dloss = (l3 + 2.0 * k3 * PHY[k]) * dPHY[k];",
                                   "double dloss = (l3 + k3 * PHY[k]) * dPHY[k];", 0),
    "phy_tangent_product_rule": ("double df1 = mu1 * LF * (dPHY[k] * M + PHY[k] * dM);",
                                 "double df1 = mu1 * LF * (PHY[k] * dM);", 0),
    "npzd_tangent_grazing_prey_term": (
        "double dG = muZ * (R * dZ[k] + Z[k] * (KP / ((KP + P[k]) * (KP + P[k]))) * dP[k]);",
        "double dG = muZ * (R * dZ[k]);", 0),
    "npzd_tangent_zooplankton_mortality": ("dmZ = 2.0 * kZ * Z[k] * dZ[k]", "dmZ = kZ * Z[k] * dZ[k]", 0),
    "npzd_tangent_sinking_through_floor": ("double dSout = (k + 1 < nlayer) ? wD * dD[k] : 0.0;",
                                           "double dSout = wD * dD[k];", 0),
    # tangent of the internal steps and of the transport
    "tangent_substep_length": ("dys[i] += ds * dq[i];", "dys[i] += dt * dq[i];", 0),
    "tangent_explicit_on_state": ("ds += a * dy[(size_t)tr * n + P->colidx[p]];",
                                  "ds += a * y[(size_t)tr * n + P->colidx[p]];", 0),
    "tangent_implicit_on_state": ("ds += bb * dz[(size_t)tr * n + s0 + k];",
                                  "ds += bb * z[(size_t)tr * n + s0 + k];", 0),
    "tangent_adds_source_not_its_tangent": ("dz[(size_t)tr * n + s0 + k] += ddq[tr * L + k];",
                                            "dz[(size_t)tr * n + s0 + k] += dq[tr * L + k];", 0),
    # reverse of the PO4-DOP term
    "ndop_reverse_martin_sign": ("Eb += qbN[k] * (pt - pb) / h[k];", "Eb += qbN[k] * (pt + pb) / h[k];", 0),
    "ndop_reverse_martin_exponent_sign": ("ub[6] += qbN[k] * E * (dpt - dpb) / h[k];",
                                          "ub[6] -= qbN[k] * E * (dpt - dpb) / h[k];", 0),
    "ndop_reverse_dop_fraction": ("double fb = Eb * (1.0 - sigma) * h[k] - qbN[k] + sigma * qbD[k];",
                                  "double fb = Eb * (1.0 - sigma) * h[k] - qbN[k] + qbD[k];", 0),
    "ndop_reverse_sigma_gradient_sign": ("ub[2] += -Eb * sumfh;", "ub[2] += Eb * sumfh;", 0),
    "ndop_reverse_attenuation_sign": ("(KI / ((I[k] + KI) * (I[k] + KI))) * (-d[k] * I[k]);",
                                      "(KI / ((I[k] + KI) * (I[k] + KI))) * (d[k] * I[k]);", 0),
    "ndop_reverse_alpha_units": ("ub[1] += fb * 360.0 * M * LF;", "ub[1] += fb * M * LF;", 0),
    "ndop_reverse_aphotic_dop_sign": ("Db[k] += lambda * (qbN[k] - qbD[k]);",
                                      "Db[k] += lambda * (qbN[k] + qbD[k]);", 0),
    # reverses of the N, PO4-DOP-PHY and NPZD-DOP terms
    "n_reverse_export_thickness": ("double fb = -qb[k] + Eb * h[k];", "double fb = -qb[k] + Eb;", 0),
    "phy_reverse_grazed_fraction": ("double f1b = -qb1[k] + (1.0 - sig3) * qb3[k] + sig3 * f3b;",
                                    "double f1b = -qb1[k] + (1.0 - sig3) * qb3[k] + f3b;", 0),
    "phy_reverse_quadratic_loss": ("PHYb[k] += lossb * (l3 + 2.0 * k3 * PHY[k]);",
                                   "PHYb[k] += lossb * (l3 + k3 * PHY[k]);", 0),
    "phy_reverse_martin_exponent_sign": ("ub[10] += qb1[k] * E * (dtop - dbot) / h[k];",
                                         "ub[10] -= qb1[k] * E * (dtop - dbot) / h[k];", 0),
    "npzd_reverse_sinking_thickness": ("double Sb = -qbD[k] / h[k] + qbD[k + 1] / h[k + 1];",
                                       "double Sb = -qbD[k] / h[k] + qbD[k + 1] / h[k];", 0),
    "npzd_reverse_zooplankton_mortality": ("Zb[k] += 2.0 * kZ * Z[k] * mZb;", "Zb[k] += kZ * Z[k] * mZb;", 0),
    "npzd_reverse_assimilation_swapped": ("double Gb = -qbP[k] + eps * qbZ[k] + (1.0 - eps) * qbO[k];",
                                          "double Gb = -qbP[k] + (1.0 - eps) * qbZ[k] + eps * qbO[k];", 0),
    "npzd_reverse_sinking_rate_units": ("ub[12] += 360.0 * D[k] * Sb;", "ub[12] += D[k] * Sb;", 0),
    "npzd_reverse_assimilation_gradient_sign": ("ub[6] += G * (qbZ[k] - qbO[k]);",
                                                "ub[6] += G * (qbO[k] - qbZ[k]);", 0),
    # reverse of the internal steps, of the transport and of the time loop
    "reverse_substep_length": ("for (int i = 0; i < len; i++) qb[i] = ds * yb[i];",
                               "for (int i = 0; i < len; i++) qb[i] = dt * yb[i];", 0),
    "reverse_increment_identity_kept": ("for (int i = 0; i < len; i++) ybar[i] += yb[i] - ybgc_bar[i];",
                                        "for (int i = 0; i < len; i++) ybar[i] += yb[i];", 0),
    "reverse_implicit_not_transposed": (
        "double bb = (1.0 - w) * B0[r * L + k] + w * B1[r * L + k];\n                    s += bb * ybar_in",
        "double bb = (1.0 - w) * B0[k * L + r] + w * B1[k * L + r];\n                    s += bb * ybar_in", 0),
    "reverse_explicit_not_transposed": (
        "ybar_out[(size_t)tr * n + P->colidx[p]] += a * zbar[(size_t)tr * n + i];",
        "ybar_out[(size_t)tr * n + i] += a * zbar[(size_t)tr * n + P->colidx[p]];", 0),
    "reverse_model_at_next_state": (
        "rc = oracle_step_adjoint(P, model, ntracer, j, states + len * j, ya,",
        "rc = oracle_step_adjoint(P, model, ntracer, j, states + len * (j + 1 < P->nstep ? j + 1 : j), ya,", 0),
    "reverse_step_index": (
        "rc = oracle_step_adjoint(P, model, ntracer, j, states",
        "rc = oracle_step_adjoint(P, model, ntracer, (j + 1) % P->nstep, states", 0),
}


def _replace_nth(text, old, new, nth):
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, "mutation site not found: %r" % old
    return text[:pos] + new + text[pos + len(old):]


def test_mutation_sites_are_in_the_derivative_code():
    """Every site lies after the last forward-model function, so no mutant touches the
    forward model (whose own pins would then catch it for the wrong reason)."""
    text = open(SRC).read()
    first_derivative = text.index("static void ndop_q_tangent(")
    for name, (old, _, nth) in MUTANTS.items():
        pos = -1
        for _ in range(nth + 1):
            pos = text.find(old, pos + 1)
        assert pos >= first_derivative, name


def _run_pins(source_text, tmp_path):
    """Build `source_text` as the oracle library and run the derivative pins against it."""
    src = tmp_path / "tmm_oracle_copy.c"
    src.write_text(source_text)
    lib = tmp_path / "liboracle_copy.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-o", str(lib), str(src), "-lm"])
    env = dict(os.environ, M3D_ORACLE_LIB=str(lib), M3D_ORACLE_THREADS="1",
               OMP_NUM_THREADS="1", OMP_WAIT_POLICY="passive")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                          [os.path.join(ROOT, "tests", p) for p in PINS],
                          env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)


@pytest.mark.slow
def test_unmutated_copy_passes_the_pins(tmp_path):
    """The control: the oracle's own source, built and loaded the same way, passes, so a
    mutant fails because of its mistake and not because of the way it is built."""
    r = _run_pins(open(SRC).read(), tmp_path)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_derivative_pins_catch_mutant(name, tmp_path):
    old, new, nth = MUTANTS[name]
    r = _run_pins(_replace_nth(open(SRC).read(), old, new, nth), tmp_path)
    assert r.returncode != 0, "the derivative pins did not catch mutant %s:\n%s" % (name, r.stdout[-2000:])
