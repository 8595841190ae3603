"""The oracle's pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/moldy_oracle.c (a dropped term, a wrong sign,
a transposed index, a wrong rounding, comparison or loop bound, a wrong function), compiles it
with the oracle's own flags, points the oracle's Python wrapper at it, and runs the pin that
should catch the mistake: the pin must fail.  An unmodified copy, built and loaded the same way, passes the same pins.  The oracle
itself is never modified: the copies live in pytest's temporary directory.
"""
import os
import sys

import pytest

import oracle
from oracle import build as oracle_build

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_pins as pins  # noqa: E402
import test_pc3_pins as pc3_pins  # noqa: E402
import test_surrogate_pins as sur_pins  # noqa: E402
import test_thermostat_pins as nvt_pins  # noqa: E402

SRC = os.path.join(os.path.dirname(oracle.__file__), "moldy_oracle.c")

# (name, text in the oracle, planted replacement, pins that must fail)
MUTANTS = [
    ("pair energy counted twice (no 1/2 on the pair sum of Eq. 1)",
     "ep += 0.5 * v;", "ep += v;",
     [lambda: pins.test_forces_are_minus_energy_gradient("fs"),
      pins.test_fs_fe_cohesive_energy_equilibrium_and_coordination]),
    ("dropped F'_j phi'_ba term of the force",
     "double g = dV + dF[i] * dphi_ab + dF[j] * dphi_ba;", "double g = dV + dF[i] * dphi_ab;",
     [lambda: pins.test_forces_are_minus_energy_gradient("fs")]),
    ("phi_ba taken with the species transposed",
     "orc_pair(pot, 1, b, a, r, &dphi_ba, &viol);", "orc_pair(pot, 1, a, b, r, &dphi_ba, &viol);",
     [lambda: pins.test_forces_are_minus_energy_gradient("fec")]),
    ("wrong sign of the pair force",
     "for (int c = 0; c < 3; c++) f[c] += gr * dv[c];", "for (int c = 0; c < 3; c++) f[c] -= gr * dv[c];",
     [lambda: pins.test_forces_are_minus_energy_gradient("cu")]),
    ("minimum image rounded down instead of to nearest",
     "return d - L * rint(d * invL);", "return d - L * floor(d * invL);",
     [pins.test_neighbour_cutoff_is_strict_and_empty_box]),
    ("list cutoff not strict",
     "if (orc_dist2(pos, i, j, L, invL, NULL) < rl2) {\n                if (c < k_max)",
     "if (orc_dist2(pos, i, j, L, invL, NULL) <= rl2) {\n                if (c < k_max)",
     [pins.test_neighbour_cutoff_is_strict_and_empty_box]),
    ("dropped term of a Hermite basis function",
     "h10 = t3 - 2.0 * t2 + t;", "h10 = t3 - 2.0 * t2;",
     [lambda: pins.test_forces_are_minus_energy_gradient("fs_tables"), pins.test_tables_reproduce_analytic_fs]),
    ("F'(rho) of Finnis-Sinclair without its factor 1/2",
     "*dF = -0.5 * A / s;", "*dF = -A / s;",
     [lambda: pins.test_forces_are_minus_energy_gradient("fs")]),
    ("dropped product-rule term of the FS pair derivative",
     "*d = 2.0 * (r - c) * q + (r - c) * (r - c) * (c1 + 2.0 * c2 * r);", "*d = 2.0 * (r - c) * q;",
     [lambda: pins.test_forces_are_minus_energy_gradient("fs")]),
    ("wrong sign of a virial component",
     "w[0] -= 0.5 * gr * dv[0] * dv[0];", "w[0] += 0.5 * gr * dv[0] * dv[0];",
     [pins.test_virial_pressure_equals_minus_dU_dV]),
    ("kinetic energy without its 1/2",
     "k += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);", "k += m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);",
     [pins.test_initial_temperature_exact_and_zero_momentum, pins.test_time_unit_matches_paper]),
    ("first half kick over a whole time step",
     "vel[3 * i + c] += half * force[3 * i + c] * im;\n                pos[3 * i + c]",
     "vel[3 * i + c] += dt_fs * force[3 * i + c] * im;\n                pos[3 * i + c]",
     [pins.test_velocity_verlet_conserves_energy_with_dt2_error, pins.test_velocity_verlet_is_time_reversible]),
    ("link-cell stencil missing its upper layer of cells",
     "for (int dz = -1; dz <= 1; dz++)\n            for (int dy = -1; dy <= 1; dy++)",
     "for (int dz = -1; dz <= 0; dz++)\n            for (int dy = -1; dy <= 1; dy++)",
     [lambda: pins.test_link_cells_equal_brute_force((3, 4, 5), 700)]),
    ("Nose-Hoover friction with the wrong sign",
     "double s = exp(-thermo[0] * h);", "double s = exp(thermo[0] * h);",
     [nvt_pins.test_extended_energy_is_conserved_with_dt2_error, nvt_pins.test_temperature_settles_at_the_target]),
    ("predictor-corrector velocity coefficient 3/4 (another scheme's) instead of 5/6",
     "c1 = 5.0 / 6.0", "c1 = 3.0 / 4.0",
     [pc3_pins.test_error_order_from_a_consistent_start_and_from_a_zero_third_derivative]),
    ("predictor without the third-derivative term of the velocity",
     "q1[k] += 2.0 * q2[k] + 3.0 * gear3[k];", "q1[k] += 2.0 * q2[k];",
     [pc3_pins.test_error_order_from_a_consistent_start_and_from_a_zero_third_derivative]),
    ("surrogate basis derivative without its Gaussian term",
     "db[k] = e * (dfc - a / w2 * fc);", "db[k] = e * dfc;",
     [sur_pins.test_surrogate_forces_are_minus_energy_gradient]),
    ("surrogate backward pass through SiLU instead of its derivative",
     "d1[p] = s * orc_dsilu(z1[p]);", "d1[p] = s * orc_silu(z1[p]);",
     [sur_pins.test_mlp_energy_and_input_gradient_match_torch_autograd]),
    ("surrogate force without the neighbour's gradient",
     "c += (grad[m * sp->nb + k] + grad[j * sp->nb + k]) * db[k];", "c += grad[m * sp->nb + k] * db[k];",
     [sur_pins.test_surrogate_forces_are_minus_energy_gradient]),
]


def _load(tmp_path, monkeypatch, old=None, new=None):
    with open(SRC) as fh:
        src = fh.read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    path = tmp_path / "moldy_oracle.c"
    path.write_text(src)
    lib = oracle_build.compile_source(str(path), str(tmp_path / "liboracle_variant.so"))
    monkeypatch.setattr(oracle_build, "build", lambda force=False: lib)
    monkeypatch.setattr(oracle, "_lib", None)


def test_unmodified_copy_passes_the_pins(tmp_path, monkeypatch):
    _load(tmp_path, monkeypatch)
    for _, _, _, checks in MUTANTS:
        for check in checks:
            check()


@pytest.mark.parametrize("name,old,new,checks", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pins(name, old, new, checks, tmp_path, monkeypatch):
    _load(tmp_path, monkeypatch, old, new)
    for check in checks:
        with pytest.raises((AssertionError, ValueError)):
            check()
