"""Plant plausible mistakes in a copy of the oracle and check that the pins catch
each one.  This shows the pins of test_oracle_pins.py constrain every part of
the oracle (equilibrium, forcing term, correction term, EOS, force stencil,
collision, streaming), not just its self-consistency.  CPU only.
"""
import pytest

import oracle as O
import test_oracle_pins as pins

# (name, text in lb_oracle.c, replacement)
MUTATIONS = [
    ("feq_drops_usq_term", "- 0.5 * usq / CS2)", ")"),
    ("guo_sign_of_u", "double emuF = (EX[i] - ux) * Fx + (EY[i] - uy) * Fy;",
     "double emuF = (EX[i] + ux) * Fx + (EY[i] + uy) * Fy;"),
    ("guo_prefactor_dropped", "double pre = 1.0 - 1.0 / (2.0 * tau_f);", "double pre = 1.0;"),
    ("correction_prefactor", "double pre = 1.0 - 1.0 / (2.0 * tau_g);",
     "double pre = 1.0 - 1.0 / tau_g;"),
    ("diagonal_weight", "w2 = 1.0 / 12.0;", "w2 = 1.0 / 6.0;"),
    ("stencil_pair_swapped", "(psi[SE] - psi[NW])", "(psi[NW] - psi[SE])"),
    ("streaming_direction",
     "d = (int64_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);\n                fn[i * N + d] = fs[i];\n"
     "                gn[i * N + d] = gs[i];",
     "d = (int64_t)wrap(y - EY[i], ny) * nx + wrap(x - EX[i], nx);\n                fn[i * N + d] = fs[i];\n"
     "                gn[i * N + d] = gs[i];"),
    ("tau_in_place_of_inverse", "(1.0 / P->tau_f) * (fl[i] - feq[i])",
     "(P->tau_f) * (fl[i] - feq[i])"),
    ("g_relaxes_with_tau_f", "(1.0 / P->tau_g) * (gl[i] - geq)",
     "(1.0 / P->tau_f) * (gl[i] - geq)"),
    ("cs_drops_eta2", "1.0 + eta + eta * eta - eta * eta * eta", "1.0 + eta - eta * eta * eta"),
    ("T_without_cv", "T[s] = e / (r * P->cv);", "T[s] = e / r;"),
    ("geq_without_cv", "double geq = P->cv * T * feq[i];", "double geq = T * feq[i];"),
    ("eq24_correction_missing", "if (P->thermal == OR_THERMAL_EQ24) gs[i] += Ci[i];", ""),
    ("psi_sq_missing_factor_2", "return 2.0 * (or_p_eos(P, rho, T_eos) - rho * CS2) / P->G;",
     "return (or_p_eos(P, rho, T_eos) - rho * CS2) / P->G;"),
    ("force_sign", "*Fx = -P->G * fx;", "*Fx = P->G * fx;"),
    ("beta_half_dropped", "fx += 0.5 * (1.0 - P->beta) * s2x;", "fx += (1.0 - P->beta) * s2x;"),
    ("no_half_force_in_u", "double ux = (mx + 0.5 * Fx) / rho;", "double ux = (mx + Fx) / rho;"),
]

# fastest first: a run stops at the first pin that fails
PINS = [
    lambda: pins.test_feq_moments(0.35, 0.03, -0.07),
    lambda: pins.test_forcing_term_moments(0.6),
    lambda: pins.test_correction_term_identities(0.8, 1.0, 0.08),
    pins.test_vdw_critical_point_closed_form,
    pins.test_cs_critical_point_published,
    pins.test_cs_virial_coefficients,
    pins.test_vdw_and_ideal_low_density_limits,
    lambda: pins.test_force_closed_form_beta0(0),
    lambda: pins.test_force_closed_form_beta0(1),
    pins.test_force_closed_form_diagonal,
    pins.test_force_taylor_limit_eq3,
    pins.test_mixed_force_linear_in_beta,
    pins.test_uniform_state_stays_uniform,
    pins.test_centre_of_mass_moves_with_momentum,
    pins.test_shear_wave_decay_viscosity,
    pins.test_thermal_diffusion_decay,
    pins.test_eq7_temperature_drift_matches_eq23,
    pins.test_eq24_removes_drift,
    pins.test_cv_scaling_exact,
    lambda: pins.test_conservation(O.THERMAL_EQ24),
    pins.test_eq24_steady_state_T_uniform,
    pins.test_eq7_steady_state_rhoT_uniform,
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new):
    src = O.source_text()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old}"
    lib = O.build_variant(src.replace(old, new), name)
    caught = None
    with O.using(lib):
        for pin in PINS:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError) as exc:
                caught = exc
                break
    assert caught is not None, f"no pin catches the planted mistake {name}"


# ---------------------------------------------------------------- cavity
import test_oracle_cavity as cav  # noqa: E402

CAVITY_MUTATIONS = [
    ("cavity_gravity_dropped", "*Fy += -rho[(int64_t)y * P->nx + x] * Cv->g_grav;", ""),
    ("cavity_isothermal_wall_adiabatic",
     "gn[o * N + s] = -gs[i] + 2.0 * OMEGA[i] * rho[s] * P->cv * Tw;", "gn[o * N + s] = gs[i];"),
    ("cavity_wall_temperatures_swapped", "double Tw = xd < 0 ? Cv->T_hot : Cv->T_cold;",
     "double Tw = xd < 0 ? Cv->T_cold : Cv->T_hot;"),
    ("cavity_anti_bounce_weight", "-gs[i] + 2.0 * OMEGA[i] * rho[s] * P->cv * Tw;",
     "-gs[i] + 2.0 * OMEGA[o] * rho[s] * P->cv * Tw + (i > 4 ? 1e-3 : 0.0);"),
    ("cavity_psi_wraps", "int xe = clampi(x + 1, nx), xw = clampi(x - 1, nx);",
     "int xe = wrap(x + 1, nx), xw = wrap(x - 1, nx);"),
]

CAVITY_PINS = [
    cav.test_uniform_state_at_wall_temperature_is_steady,
    cav.test_mass_conserved_and_gravity_stratifies,
    cav.test_conduction_nusselt_is_one,
]


@pytest.mark.parametrize("name,old,new", CAVITY_MUTATIONS, ids=[m[0] for m in CAVITY_MUTATIONS])
def test_planted_cavity_mistake_is_caught(name, old, new):
    src = O.source_text()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old}"
    lib = O.build_variant(src.replace(old, new), name)
    caught = None
    with O.using(lib):
        for pin in CAVITY_PINS:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError) as exc:
                caught = exc
                break
    assert caught is not None, f"no cavity pin catches the planted mistake {name}"


# ------------------------------------------------- FD treatment with walls
import test_oracle_channel as chan  # noqa: E402

WALL_FD_MUTATIONS = [
    ("fd_cavity_side_wall_not_reflected", "Xn[i] = 2.0 * Tw - X[m];", "Xn[i] = X[m];"),
    ("fd_channel_inlet_ghost_mirrored", "if (xn < 0) return 2.0 * Ch->T_in - Xm;", "if (xn < 0) return Xm;"),
    ("fd_channel_plate_ghost_sign", "return 2.0 * Ch->T_w - Xm;", "return 2.0 * Ch->T_w + Xm;"),
]

WALL_FD_PINS = [
    lambda: chan.test_fd_table1_fully_developed_nusselt("A"),
    cav.test_fd_cavity_table2_ra1e3,
]


@pytest.mark.parametrize("name,old,new", WALL_FD_MUTATIONS, ids=[m[0] for m in WALL_FD_MUTATIONS])
def test_planted_wall_fd_mistake_is_caught(name, old, new):
    src = O.source_text()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old}"
    lib = O.build_variant(src.replace(old, new), name)
    caught = None
    with O.using(lib):
        for pin in WALL_FD_PINS:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError) as exc:
                caught = exc
                break
    assert caught is not None, f"no pin catches the planted mistake {name}"


# ------------------------------------------------------- start at rest
import test_oracle_init as ini  # noqa: E402

INIT_MUTATIONS = [
    ("init_velocity_sign", "double vx = -Fx / (2.0 * rho0[s]);", "double vx = Fx / (2.0 * rho0[s]);"),
    ("init_velocity_half_missing", "double vy = -Fy / (2.0 * rho0[s]);", "double vy = -Fy / rho0[s];"),
    ("init_psi_from_T_psi", "psi2[s] = or_psi_sq(P, rho0[s], T0[s]);",
     "psi2[s] = or_psi_sq(P, rho0[s], P->T_psi);"),
    ("init_g_without_T",
     "or_feq(rho0[s], vx, vy, feq);\n            for (int i = 0; i < 9; ++i) {\n"
     "                f[i * N + s] = feq[i];\n                g[i * N + s] = P->cv * T0[s] * feq[i];",
     "or_feq(rho0[s], vx, vy, feq);\n            for (int i = 0; i < 9; ++i) {\n"
     "                f[i * N + s] = feq[i];\n                g[i * N + s] = P->cv * feq[i];"),
    ("init_g_east_scaled", "g[i * N + s] = P->cv * T0[s] * feq[i];\n            }\n        }\n    }\n    free(psi); free(psi2);",
     "g[i * N + s] = P->cv * T0[s] * feq[i] * (i == 1 ? 1.001 : 1.0);\n            }\n        }\n    }\n"
     "    free(psi); free(psi2);"),
]

INIT_PINS = [ini.test_balanced_start_of_uniform_state_is_plain_equilibrium] + [
    (lambda c=c: ini.test_balanced_start_is_at_rest(*c)) for c in ini.CASES] + [
    (lambda c=c: ini.test_balanced_start_keeps_rho_and_T(*c)) for c in ini.CASES]


@pytest.mark.parametrize("name,old,new", INIT_MUTATIONS, ids=[m[0] for m in INIT_MUTATIONS])
def test_planted_init_mistake_is_caught(name, old, new):
    src = O.source_text()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old}"
    lib = O.build_variant(src.replace(old, new), name)
    caught = None
    with O.using(lib):
        for pin in INIT_PINS:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError) as exc:
                caught = exc
                break
    assert caught is not None, f"no pin catches the planted mistake {name}"
