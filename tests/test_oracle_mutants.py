"""Planted mistakes in the oracle must fail its pins.

Each case edits one expression of ``oracle/cascade_oracle.c`` in a temporary
copy (a dropped term, a wrong sign or index, a swapped operand), compiles it,
and runs the pins of ``test_oracle_pins.py`` against that build: at least one
pin must fail.  The unmodified source must pass the same pins, so a failure is
the mutation's doing.  All of this runs on the CPU.
"""
import os

import pytest

import oracle
import test_oracle_corotating as corot
import test_oracle_pins as pins

ALL_PINS = [
    pins.test_philox_known_answers,
    pins.test_seed_normals_are_standard_normal,
    pins.test_quiet_start_layout_and_gauss,
    pins.test_single_particle_uniform_field_second_order,
    pins.test_electron_moves_against_field,
    pins.test_gauss_and_charge_conservation_with_qed,
    pins.test_mean_current_and_field_of_a_hand_built_state,
    pins.test_cold_uniform_mode_frequency,
    pins.test_relativistic_uniform_mode_period,
    pins.test_standing_langmuir_wave,
    pins.test_energy_conservation_with_cascade,
    pins.test_single_emission_bookkeeping,
    pins.test_electron_emission_runs_backwards,
    pins.test_multi_photon_emission_conserves_energy,
    pins.test_threshold_tie_emits,
    pins.test_in_place_conversion,
    lambda lib=None: pins.test_frozen_field_growth_rate(0.1, lib),
    corot.test_background_current_drives_the_uniform_mode,
    corot.test_corotating_equilibrium_is_stationary,
    corot.test_open_boundary_removes_departing_particles,
    corot.test_open_boundary_outflow_keeps_gauss,
    corot.test_open_boundary_gather_uses_the_edge_field,
    corot.test_open_boundary_drops_photons_converting_outside,
]

# (name, original text, mutated text)
MUTANTS = [
    ("philox_multiplier", "0xCD9E8D57u * (uint64_t)c[2]", "0xCD9E8D55u * (uint64_t)c[2]"),
    ("philox_key_bump", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE84u;"),
    ("box_muller_branch", "*z_posi = rad * sin(ang);", "*z_posi = rad * cos(ang);"),
    ("quiet_start_offset", "double off = ((double)k + 0.5) / (double)p->ppc;",
     "double off = ((double)k + 0.25) / (double)p->ppc;"),
    ("gather_weights_swapped", "double Ep = (1.0 - w) * s->E[ia] + w * s->E[ib];",
     "double Ep = w * s->E[ia] + (1.0 - w) * s->E[ib];"),
    ("gather_left_weight", "ib = c; w = o + 0.5; }", "ib = c; w = 0.5 - o; }"),
    ("push_charge_dropped", "double u = s->u[p] + q * dt * Ep;", "double u = s->u[p] + dt * Ep;"),
    ("move_uses_momentum", "double d = u / g * dtdx;", "double d = u * dtdx;"),
    ("deposit_sign", "S[c] += q * (o2 - o);", "S[c] += q * (o - o2);"),
    ("deposit_crossing_edge", "S[c2] += q * o2;", "S[c] += q * o2;"),
    ("deposit_backward_term", "S[c2] += q * (o2 - 1.0);", "S[c2] += q * (1.0 - o2);"),
    ("ampere_sign", "s->E[i] = s->E[i] - dt * (s->J[i] - s->p.j_m);", "s->E[i] = s->E[i] + dt * (s->J[i] - s->p.j_m);"),
    ("current_scale", "s->jscale = p->n0 * p->dx / ((double)p->ppc * p->dt);",
     "s->jscale = 2.0 * p->n0 * p->dx / ((double)p->ppc * p->dt);"),
    ("recoil_dropped", "double g2 = g - (double)k * eps;", "double g2 = g;"),
    ("single_photon_only", "int64_t k = 1 + (int64_t)floor((g - thr) / eps);", "int64_t k = 1;"),
    ("threshold_strict", "if (!(g >= thr)) continue;", "if (!(g > thr)) continue;"),
    ("pair_gets_full_energy", "const double h = 0.5 * s->p.eps_gamma;", "const double h = s->p.eps_gamma;"),
    ("flight_one_step_short", "const int64_t conv = s->step + 1 + s->n_pp;", "const int64_t conv = s->step + s->n_pp;"),
    ("photon_flies_backwards", "oc = s->off[p] + s->lpp_frac;", "oc = s->off[p] - s->lpp_frac;"),
    ("photon_direction_lost", "s->ph_dir[s->nph] = (int8_t)(sgn > 0 ? 1 : -1);", "s->ph_dir[s->nph] = 1;"),
    ("kinetic_energy_weight", "uk += s->w * s->gam[p];", "uk += s->gam[p];"),
    ("field_energy_half", "ue += 0.5 * s->E[i] * s->E[i] * s->p.dx;", "ue += s->E[i] * s->E[i] * s->p.dx;"),
    ("mean_current_half", "d->J_mean = sj / nx;", "d->J_mean = 0.5 * sj / nx;"),
    ("field_max_from_edge_0", "double a = fabs(s->E[i]);", "double a = fabs(s->E[0]);"),
    ("field_max_signed", "double a = fabs(s->E[i]);", "double a = s->E[i];"),
    ("background_current_sign", "s->E[i] = s->E[i] - dt * (s->J[i] - s->p.j_m);",
     "s->E[i] = s->E[i] - dt * (s->J[i] + s->p.j_m);"),
    ("background_charge_sign", "(s->rho_dx[i] - s->p.rho_gj * s->p.dx)", "(s->rho_dx[i] + s->p.rho_gj * s->p.dx)"),
    ("open_gather_wraps", "ia = (c == 0) ? (open ? 0 : nx - 1) : c - 1;", "ia = (c == 0) ? nx - 1 : c - 1;"),
    ("departing_deposit", "S[c] += q * (1.0 - o);", "S[c] += q * (0.5 - o);"),
    ("photon_outside_kept", "if (s->p.open_bc && (ci < 0 || ci >= s->p.nx)) continue;", "if (0) continue;"),
]


@pytest.fixture(scope="module")
def build_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


def _build(src_text, build_dir, name):
    src = os.path.join(build_dir, f"{name}.c")
    with open(src, "w") as f:
        f.write(src_text)
    return oracle.compile_source(src, os.path.join(build_dir, f"lib{name}.so"))


def _failing_pins(lib, stop_at_first=True):
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib=lib)
        except (AssertionError, oracle.OracleError, ValueError, ZeroDivisionError, FloatingPointError):
            failed.append(getattr(pin, "__name__", "pin"))
            if stop_at_first:
                break
    return failed


def test_unmodified_copy_passes_all_pins(build_dir):
    src = open(oracle.SOURCE).read()
    lib = _build(src, build_dir, "unmodified")
    assert _failing_pins(lib, stop_at_first=False) == []


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, orig, mut, build_dir):
    src = open(oracle.SOURCE).read()
    assert src.count(orig) == 1, f"mutation site for {name} not unique"
    lib = _build(src.replace(orig, mut), build_dir, name)
    assert _failing_pins(lib), f"no pin caught mutation {name}"
