"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle's C source (the parameter
beta, the snapshot index, a mass weight, the Hamming distance, the damping
factor, the window argument, a forcing sign, a Givens conjugate, the sign of
the damping term, the projection phase, the I_abd damping weight, the stencil
family's mass and stiffness mixes, the adjoint source of the misfit gradient,
a term of the recurrence adjoint, the phase of the exact run's forcing),
builds it, runs a battery of the pins of
test_oracle_pins.py, test_oracle_abd.py and test_oracle_gradient.py against
it, and requires that at least one pin fails.  The
unmodified source passes the same battery.  Everything runs on the CPU.
"""
import os

import pytest

import oracle
import test_oracle_abd as abd
import test_oracle_gradient as grad
import test_oracle_pins as pins

# (name, original text, planted text): each original occurs in the source; the
# first occurrence is replaced
MUTANTS = [
    ("beta", "out->beta = x / sin(x);", "out->beta = x / tan(x);"),
    ("snapshot index", "long long j_im = nsteps - q->nP / 4;",
     "long long j_im = nsteps - q->nP / 2;"),
    ("mass weight", "M[1] = 0.5 * (2.0 / 36.0);", "M[1] = 0.5 * (1.0 / 36.0);"),
    ("Hamming distance", "int s = popcount_small((unsigned)(b ^ g));",
     "int s = popcount_small((unsigned)(b & g));"),
    ("damping factor", "/ (1.0 + 0.5 * L);", "/ (1.0 + L);"),
    ("window argument", "ora_window(1.0 - (double)j / (double)nsteps, q->rho)",
     "ora_window((double)j / (double)nsteps, q->rho)"),
    ("forcing sign", "f[i] = chi * (cs * creal(F[i]) - sn * cimag(F[i]));",
     "f[i] = chi * (cs * creal(F[i]) + sn * cimag(F[i]));"),
    ("Givens conjugate", "col[j] = conj(cs[j]) * a + sn[j] * b;",
     "col[j] = cs[j] * a + sn[j] * b;"),
    ("damping sign", "out[i] += -t[2 * i + 1] + I * t[2 * i];",
     "out[i] += t[2 * i + 1] - I * t[2 * i];"),
    ("projection phase", "cplx e = cos(th) - I * sin(th);", "cplx e = cos(th) + I * sin(th);"),
    ("I_abd damping weight", "(1.0 - cos(q->omega * q->dt)) / q->alpha / q->omega;",
     "(1.0 + cos(q->omega * q->dt)) / q->alpha / q->omega;"),
    ("family mass mix", "M[s] = a * mc[s] + (1.0 - a) * (s == 0 ? lumped : 0.0);",
     "M[s] = (1.0 - a) * mc[s] + a * (s == 0 ? lumped : 0.0);"),
    ("adjoint source", "r[rec_idx[k]] += conj(res);", "r[rec_idx[k]] += res;"),
    ("recurrence adjoint R term", "grad_R[i] += cR * lk[i] * (uk[i] - uk2[i]);",
     "grad_R[i] += cR * lk[i] * (uk[i] + uk2[i]);"),
    ("exact-run forcing phase", "cplx e = cexp(I * q->omega * t);",
     "cplx e = cexp(-I * q->omega * t);"),
    ("family stiffness mix", "S[s] = gamma * sq1[s] + (1.0 - gamma) * sfd[s];",
     "S[s] = gamma * sq1[s] + (1.0 - gamma) * sq1[s];"),
    ("window kinked at its ends", "    return v * v;\n}", "    return v;\n}"),
]

BATTERY = [
    lambda: pins.test_q1mix_tables_are_q1_element_matrices(2),
    lambda: pins.test_q1mix_tables_are_q1_element_matrices(3),
    lambda: pins.test_fd5_constant_k_is_the_papers_5_point_operator(2),
    lambda: pins.test_sine_modes_diagonalise_constant_coefficient_operator(2, "q1mix"),
    lambda: pins.test_sine_modes_diagonalise_constant_coefficient_operator(3, "q1mix"),
    lambda: pins.test_parameter_formulas(),
    lambda: pins.test_window_is_admissible(),
    lambda: pins.test_prop1_time_harmonic_solutions_are_reproduced_exactly(2, (13, 11)),
    lambda: pins.test_theorem1_energy_identity(),
    lambda: pins.test_preconditioner_on_sine_mode_equals_greens_sum(2, "q1mix", "zero", "table1"),
    lambda: pins.test_preconditioner_on_sine_mode_equals_greens_sum(2, "q1mix", 40.0, "table1"),
    lambda: pins.test_preconditioner_on_sine_mode_equals_greens_sum(2, "q1mix", 40.0, "exact"),
    lambda: pins.test_direct_solve_matches_scipy(2, (23, 19)),
    lambda: pins.test_gmres_unpreconditioned_matches_scipy_residual_history(),
    lambda: pins.test_gmres_recovers_manufactured_solution("fgmres", "table1"),
    lambda: pins.test_gmres_recovers_manufactured_solution("left", "exact"),
    lambda: pins.test_projection_recovers_time_harmonic_amplitude(8, 2, 37),
    lambda: pins.test_projection_on_sine_mode_equals_greens_sum(2, "q1mix", "zero", 1),
    lambda: pins.test_family_tables_mix_q1_element_matrices_and_edge_stiffness(2, 0.3, 0.6),
    lambda: abd.test_abd_reproduces_time_harmonic_solutions_exactly(2, (9, 8), "node"),
    lambda: abd.test_abd_energy("layer"),
    lambda: abd.test_cell_damping_operator("q1mix"),
    lambda: pins.test_sine_modes_diagonalise_family_operator(2, 0.3, 0.6),
    lambda: grad.test_gradient_matches_central_differences(2, (11, 9)),
    lambda: grad.test_recurrence_gradient_matches_central_differences(2, (11, 9), "table1"),
    lambda: pins.test_theorem5_rate_of_ST_on_sine_modes((8, 1)),
]


def failing_pins(lib_path):
    failed = []
    with oracle.use_library(lib_path):
        for k, pin in enumerate(BATTERY):
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                failed.append(k)
    return failed


def build_variant(tmp_path, name, old, new):
    src = open(oracle.source_path()).read()
    assert old in src, name
    path = os.path.join(str(tmp_path), "ora_" + name.replace(" ", "_"))
    with open(path + ".c", "w") as f:
        f.write(src.replace(old, new, 1))
    return oracle.compile_library(path + ".c", path + ".so")


def test_unmodified_oracle_passes_the_battery(tmp_path):
    lib = build_variant(tmp_path, "same", "#include <math.h>", "#include <math.h>")
    assert failing_pins(lib) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    lib = build_variant(tmp_path, name, old, new)
    assert failing_pins(lib), f"no pin catches: {name}"


def test_rate_pin_alone_catches_a_kinked_window(tmp_path):
    """The Theorem 5 rate pin by itself catches a window that keeps the limit
    S_T -> H^-1 but is only continuous (sin instead of sin^2 on the taper: a
    kink where the taper meets 0 and 1), whose error decays like T^-1."""
    name, old, new = next(m for m in MUTANTS if m[0] == "window kinked at its ends")
    lib = build_variant(tmp_path, name, old, new)
    with oracle.use_library(lib):
        with pytest.raises(AssertionError):
            pins.test_theorem5_rate_of_ST_on_sine_modes((8, 1))
