"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU only), in the
forward model, builds it, and runs the pin suite against it: the suite must fail for
every mutant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tmm_oracle.c")

MUTANTS = {
    "interp_weights_swapped": ("(1.0 - w) * a0[p] + w * a1[p]", "w * a0[p] + (1.0 - w) * a1[p]"),
    "block_transposed": ("B0[r * L + k] + w * B1[r * L + k]", "B0[k * L + r] + w * B1[k * L + r]"),
    "q_on_explicit_result": ("ycol[tr * L + k] = y[(size_t)tr * n + s0 + k]", "ycol[tr * L + k] = z[(size_t)tr * n + s0 + k]"),
    "dop_remin_dropped_in_euphotic": ("qN[k] = -f + lambda * DOP[k];", "qN[k] = -f;"),
    "martin_sign": ("(Ftop - Fbot) / h[k]", "(Fbot - Ftop) / h[k]"),
    "export_fraction": ("E += (1.0 - sigma) * f * h[k];", "E += sigma * f * h[k];"),
    "bottom_deposit_dropped": ("(k == nlayer - 1) ? 0.0 : E * pow(zbot / zeu, -b)", "E * pow(zbot / zeu, -b)"),
    "light_at_wrong_depth": ("exp(-d[k] * kw)", "exp(-h[k] * kw)"),
    "alpha_units": ("u[1] * 360.0", "u[1]"),
    "insolation_term": ("cos(phi) * cos(delta) * sin(h0)", "cos(phi) * cos(delta) * cos(h0)"),
    "month_index": ("*m1 = (mk + 1) % nmonth;", "*m1 = (mk + 2) % nmonth;"),
    "forcing_time": ("double t = (double)j / P->nstep;", "double t = (double)(j + 1) / P->nstep;"),
    "substep_length": ("double ds = dt / nsub;", "double ds = dt;"),
    "csr_gather": ("y[(size_t)tr * n + P->colidx[p]]", "y[(size_t)tr * n + i]"),
    "euphotic_layers": ("int neu = nlayer < 2 ? nlayer : 2;", "int neu = nlayer < 3 ? nlayer : 3;"),
    "light_half_saturation": ("(I / (I + KI))", "(I / (I + KN))"),
    "declination_phase": ("cos(2.0 * pi * (t + 10.0 / 360.0))", "cos(2.0 * pi * (t - 10.0 / 360.0))"),
    # the N, PO4-DOP-PHY and NPZD-DOP models
    "n_export_dropped": ("E += f * h[k];", "E += 0.5 * f * h[k];"),
    "n_martin_exponent": ("double top = pow(ztop / zeu, -b);", "double top = pow(ztop / zeu, b);"),
    "phy_grazed_fraction": ("double f3 = sig3 * f1;", "double f3 = f1;"),
    "phy_growth_without_phy": ("double f1 = mu1 * PHY[k]", "double f1 = mu1"),
    "phy_quadratic_loss_sign": ("q3[k] = (1.0 - sig3) * f1 - loss - l3p * PHY[k];",
                                "q3[k] = (1.0 - sig3) * f1 + loss - l3p * PHY[k];"),
    "npzd_assimilation": ("q[2 * nlayer + k] = eps * G - mZ - eZ;", "q[2 * nlayer + k] = G - mZ - eZ;"),
    "npzd_sinking_through_floor": ("(k + 1 < nlayer) ? wD * D[k] : 0.0", "wD * D[k]"),
    "npzd_grazing_not_saturating": ("(P[k] / (KP + P[k]))", "(P[k] / KP)"),
    "npzd_growth_below_euphotic": ("        if (k < neu) {\n            double I", "        if (k < nlayer) {\n            double I"),
}


def _run_pins(source_text, tmp_path):
    """Build `source_text` as the oracle library and run the forward pins against it."""
    mutated = tmp_path / "tmm_oracle_mut.c"
    mutated.write_text(source_text)
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-o", str(lib), str(mutated), "-lm"])
    env = dict(os.environ, M3D_ORACLE_LIB=str(lib), M3D_ORACLE_THREADS="1",
               OMP_NUM_THREADS="1", OMP_WAIT_POLICY="passive")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                           os.path.join(ROOT, "tests", "test_oracle_models.py")],
                          env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)


@pytest.mark.slow
def test_unmutated_copy_passes_the_pins(tmp_path):
    """The control: the oracle's own source, built and loaded as the mutants are, passes."""
    r = _run_pins(open(SRC).read(), tmp_path)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert old in text, "mutation site not found: %s" % name
    # the first occurrence is in the forward model (its tangent and adjoint follow later)
    r = _run_pins(text.replace(old, new, 1), tmp_path)
    assert r.returncode != 0, "the pins did not catch mutant %s:\n%s" % (name, r.stdout[-2000:])
