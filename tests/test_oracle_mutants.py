"""The pins have teeth: copies of the oracle with one plausible mistake
planted (a sign, a side, an index, a skipped term in the shear-wave branch
of the Riemann solver, the reflective ghosts, the 3D tangential loop, the
totals' cell volume, the rule for a contact at rest, the void-opening
modifier's tension test, critical-damage test, surface speed, gap volume,
mass flux and the void's share of the stress, the seeding; the cold and
shear pressures, the Steinberg modulus and Grueneisen derivative, the
Hencky strain, the perturbed yield stress, the return factor and
equivalent stress, the unimodular normalisation, the RK4 weights, the
Bonora exponent, the rate term, the triaxiality and the lattice weights,
damage in compression, the simple law's 1 - D, the hardening exponent, the
strength kept at critical damage, four powers of the threshold strain;
the mixture's 1/Gamma weights, mass weights, Gamma' term and shear part
of the sound speed; the half step's length, the limiter, the slope's sign,
the signs of the non-conservative terms of Fbar, phi and the update, X's
term dropped, the CFL speed without c_L, the WENO3 weights, the Riemann
solver's wave speed, star speed and star side, the physical flux's stress
sign, stress row, Fbar row and history transport, the time step from the
largest spacing, a phase-density bound of 2 for e, the RK3 stage weights
and stage order, the WENO3 left candidate; the fragment labelling's
periodic faces, cut-off side, critical-damage exclusion, solid-only mass and
neighbour stride) are each caught by at least one check of
tests/pins_sources.py, tests/pins_fragments.py, tests/pins_step.py,
tests/pins_void.py or tests/pins_waves.py.  Each copy is compiled to a
temporary library and checked in a child process.  CPU only."""
import concurrent.futures as cf
import functools
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402

# (name, text in mmfrac_oracle.c, replacement): each text occurs exactly once
MUTANTS = [
    ("shear_row_sign",
     "Us[g->o_F + c] + sgn * aK->F[3 * d + j] * du / csK",
     "Us[g->o_F + c] - sgn * aK->F[3 * d + j] * du / csK"),
    ("shear_star_density_side",
     "const double rsK = left ? rsL : rsR;",
     "const double rsK = left ? rsR : rsL;"),
    ("shear_energy_sign",
     "Uss[g->o_E] += sgn * (tss * uss - tauK * uKt) / csK;",
     "Uss[g->o_E] -= sgn * (tss * uss - tauK * uKt) / csK;"),
    ("shear_impedance_swap",
     "const double uss = (tauR - tauL + ZL * uLt + ZR * uRt) / (ZL + ZR);",
     "const double uss = (tauR - tauL + ZR * uLt + ZL * uRt) / (ZL + ZR);"),
    ("shear_tangential_z_skipped",
     "for (int t = 0; t < g->dim; ++t) {\n    if (t == d) continue;\n    const double uLt",
     "for (int t = 0; t < 2 && t < g->dim; ++t) {\n    if (t == d) continue;\n    const double uLt"),
    ("mirror_flips_diagonal_too",
     "if ((i == d) != (j == d)) u[g->o_F + c] = -u[g->o_F + c];",
     "if ((i == d) || (j == d)) u[g->o_F + c] = -u[g->o_F + c];"),
    ("mirror_keeps_normal_velocity",
     "u[g->o_mom + d] = -u[g->o_mom + d];",
     "u[g->o_mom + d] = u[g->o_mom + d];"),
    ("mirror_keeps_X",
     "u[g->o_X + d] = 2.0 * wall - u[g->o_X + d];",
     "u[g->o_X + d] = u[g->o_X + d];"),
    ("reflective_ghost_order",
     "src = side == 0 ? m : n - 1 - m;",
     "src = side == 0 ? 1 - m : n - 2 + m;"),
    ("totals_cubic_cells",
     "double dV = 1.0;\n  for (int k = 0; k < g->dim; ++k) dV *= g->dx[k];\n  const int nq",
     "double dV = 1.0;\n  for (int k = 0; k < g->dim; ++k) dV *= g->dx[0];\n  const int nq"),
    ("contact_at_rest_takes_one_side",
     "if (fabs(Ss) <= 16.0 * DBL_EPSILON * (SR - SL)) {",
     "if (0) {"),
    ("void_opens_in_compression",
     "aL->sig[3 * d + d] + aR->sig[3 * d + d] > 0.0) {",
     "aL->sig[3 * d + d] + aR->sig[3 * d + d] < 0.0) {"),
    ("void_opens_without_critical_damage",
     "return is_damaged(m) && D >= m->D_crit * (1.0 - 1e-4);",
     "return is_damaged(m) && D >= 0.9 * m->D_crit;"),
    ("critical_damage_without_rounding_margin",
     "return is_damaged(m) && D >= m->D_crit * (1.0 - 1e-4);",
     "return is_damaged(m) && D >= m->D_crit;"),
    ("free_surface_speed_sign",
     "return a->u[d] + a->sig[3 * d + d] / (a->rho * (SK - a->u[d]));",
     "return a->u[d] - a->sig[3 * d + d] / (a->rho * (SK - a->u[d]));"),
    ("gap_void_sign",
     "Fo[g->o_phi + g->void_l] += ufs[side] - ufc;",
     "Fo[g->o_phi + g->void_l] -= ufs[side] - ufc;"),
    ("gap_side_takes_own_mass_flux",
     "        for (int k = 0; k < nf; ++k) Fo[k] = Fc[k];\n        for (int c = 0; c < g->nF; ++c)",
     "        for (int k = 0; k < nf; ++k) Fo[k] = Fs[side][k];\n        for (int c = 0; c < g->nF; ++c)"),
    ("void_energy_in_closure",
     "    if (is_void(&g->mat[l])) continue; /* no energy, no part in the closure */\n",
     ""),
    ("seed_probe_into_the_void",
     "p[d] = cc[d] + 1.5 * h * (-gr[d] / gn);",
     "p[d] = cc[d] + 1.5 * h * (gr[d] / gn);"),
    ("seed_offset_sign",
     "Xn[(size_t)k * g->ncell + c] = Xi[k] - (p[k] - cc[k]);",
     "Xn[(size_t)k * g->ncell + c] = Xi[k] + (p[k] - cc[k]);"),
    ("seed_weights_swapped",
     "w *= b ? f[d] : 1.0 - f[d];",
     "w *= b ? 1.0 - f[d] : f[d];"),
    ("seed_periodic_without_shift",
     "*shift = side == 0 ? -(g->hi[d] - g->lo[d]) : (g->hi[d] - g->lo[d]);",
     "*shift = 0.0;"),
    ("seed_mirror_ignored",
     "if (mirror[k]) x = 2.0 * wall[k] - x;",
     ""),
    ("seed_threshold_inverted",
     "if (!(void_at(g, ix) > 0.5)) continue;",
     "if (!(void_at(g, ix) < 0.5)) continue;"),
    # closures, Hencky strain, plastic return, damage, lookup (pins_sources.py)
    ("cold_pressure_sign",
     "const double pc = psi * m->K0 / (2.0 * a * a) * (2.0 * a * q * ea - q * q);",
     "const double pc = psi * m->K0 / (2.0 * a * a) * (2.0 * a * q * ea + q * q);"),
    ("shear_pressure_exponent",
     "const double ps = m->beta * G * J2;",
     "const double ps = (m->beta + 1.0) * G * J2;"),
    ("steinberg_dG_sign",
     "const double q1 = u * (pc1 - pc0 / (3.0 * rho));",
     "const double q1 = u * (pc1 + pc0 / (3.0 * rho));"),
    ("grueneisen_derivative_sign",
     "out[5] = (-m->Gamma1 * u / 3.0 - m->gamma_s * m->Gamma2 * g2) / Gam;",
     "out[5] = (-m->Gamma1 * u / 3.0 + m->gamma_s * m->Gamma2 * g2) / Gam;"),
    ("hencky_without_half",
     "for (int k = 0; k < 3; ++k) h[k] = 0.5 * log(lam[k]);",
     "for (int k = 0; k < 3; ++k) h[k] = log(lam[k]);"),
    ("yield_without_perturbation",
     "const double wgt = phi[l] * phihat * psi;",
     "const double wgt = phi[l] * psi;"),
    ("return_factor_2G",
     "const double k = (str - 3.0 * Gm * dl) / str;",
     "const double k = (str - 2.0 * Gm * dl) / str;"),
    ("equivalent_stress_factor",
     "const double str = sqrt(6.0) * Gm * J;",
     "const double str = sqrt(3.0) * Gm * J;"),
    ("det_not_renormalised",
     "const double dt3 = cbrt(det3(F));",
     "const double dt3 = 1.0;"),
    ("rk4_drops_k3",
     "double Dn = D + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);",
     "double Dn = D + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k2 + k4);"),
    ("bonora_exponent",
     "pow(Dc - D, (aD - 1.0) / aD)",
     "pow(Dc - D, (aD - 1.0))"),
    ("rate_log_inverted",
     "const double r = 1.0 + m->c3 * log(dl / (dt * m->edot0));",
     "const double r = 1.0 + m->c3 * log(dt * m->edot0 / dl);"),
    ("lookup_weights_swapped",
     "wt *= b ? w[k] : 1.0 - w[k];",
     "wt *= b ? 1.0 - w[k] : w[k];"),
    ("triaxiality_poisson_factor",
     "3.0 * (1.0 - 2.0 * poisson) * (rho0 / rho) * (x * x);",
     "3.0 * (1.0 - poisson) * (rho0 / rho) * (x * x);"),
    # the physical flux (pins_step.py)
    ("momentum_flux_stress_sign",
     "    f[g->o_mom + k] = u[g->o_mom + k] * ud - ax->sig[3 * k + d];",
     "    f[g->o_mom + k] = u[g->o_mom + k] * ud + ax->sig[3 * k + d];"),
    ("energy_flux_stress_row",
     "              (ax->sig[3 * d + 0] * ax->u[0] + ax->sig[3 * d + 1] * ax->u[1] +",
     "              (ax->sig[3 * d + 0] * ax->u[0] + ax->sig[3 * d + 1] * ax->u[0] +"),
    ("fbar_flux_row",
     "                             : u[g->o_F + c] * ud - ax->F[3 * d + j] * ax->u[i];",
     "                             : u[g->o_F + c] * ud - ax->F[3 * i + j] * ax->u[d];"),
    ("history_not_advected",
     "  for (int k = 0; k < 2 * g->nhist; ++k) f[g->o_hist + k] = u[g->o_hist + k] * ud;",
     "  for (int k = 0; k < 2 * g->nhist; ++k) f[g->o_hist + k] = 0.0;"),
    ("cfl_largest_spacing",
     "    if (g->dx[k] < dxm) dxm = g->dx[k];",
     "    if (g->dx[k] > dxm) dxm = g->dx[k];"),
    ("phase_bound_factor_two",
     "  const double e = 2.718281828459045;\n  for (int l = 0; l < g->nmat; ++l) {\n    const double r0 = w_rec",
     "  const double e = 2.0;\n  for (int l = 0; l < g->nmat; ++l) {\n    const double r0 = w_rec"),
    ("rk3_second_stage_weights",
     "      X2[q] = 0.75 * X0[q] + 0.25 * (X1[q] + dt * x_rhs(g, X1, vel, c, k));",
     "      X2[q] = 0.5 * X0[q] + 0.5 * (X1[q] + dt * x_rhs(g, X1, vel, c, k));"),
    ("rk3_last_stage_from_X1",
     "      Xn[q] = (1.0 / 3.0) * X0[q] + (2.0 / 3.0) * (X2[q] + dt * x_rhs(g, X2, vel, c, k));",
     "      Xn[q] = (1.0 / 3.0) * X0[q] + (2.0 / 3.0) * (X2[q] + dt * x_rhs(g, X1, vel, c, k));"),
    ("weno3_left_candidate",
     "  const double q0 = -0.5 * a + 1.5 * b;",
     "  const double q0 = 0.5 * a + 0.5 * b;"),
    # fragment labelling (pins_fragments.py)
    ("fragment_periodic_ignored",
     "            if (g->bc[d][side] != OR_BC_PERIODIC) continue;",
     "            continue;"),
    ("fragment_cut_off_side",
     "  return phis > 1.0 - theta;",
     "  return phis > theta;"),
    ("fragment_critical_kept",
     "      if (is_critical(&g->mat[l], U[(size_t)(g->o_hist + 2 * h + 1) * n + c] / arho)) return 0;",
     "      if (is_critical(&g->mat[l], U[(size_t)(g->o_hist + 2 * h + 1) * n + c] / arho)) (void)0;"),
    ("fragment_mass_with_gas",
     "      for (int l = 0; l < g->nmat; ++l) {\n        if (g->mat[l].eos != 1) continue;\n        const double y",
     "      for (int l = 0; l < g->nmat; ++l) {\n        const double y"),
    ("fragment_neighbours_along_x_only",
     "          const long nb = c + (j - i) * stride;",
     "          const long nb = c + (j - i);"),
    # damage gate and laws, hardening, strength at critical damage (pins_sources.py)
    ("damage_in_compression",
     "  if (!(p < 0.0) || !(eps > thresh)) return 0.0;",
     "  if (!(eps > thresh)) return 0.0;"),
    ("simple_damage_without_1_minus_D",
     "  if (m->damage == 2) return m->Ddot0 * (1.0 - D) * epsdot;",
     "  if (m->damage == 2) return m->Ddot0 * epsdot;"),
    ("hardening_exponent_inverted",
     "      hard += m->c2 * pow(e, m->n_hard);",
     "      hard += m->c2 * pow(e, 1.0 / m->n_hard);"),
    ("critical_keeps_strength",
     "    if (is_critical(m, D[l])) continue;\n    const double psi = is_damaged(m) ? 1.0 - D[l] : 1.0;\n    /* advection",
     "    const double psi = is_damaged(m) ? 1.0 - D[l] : 1.0;\n    /* advection"),
    ("threshold_Rt_power",
     "  return pow(eps_t, 1.0 / Rt) / pow(Rt, 1.0 / n) * pow(num / den, 1.0 / (2.0 * n));",
     "  return pow(eps_t, 1.0 / Rt) / pow(Rt, n) * pow(num / den, 1.0 / (2.0 * n));"),
    ("threshold_eps_power",
     "  return pow(eps_t, 1.0 / Rt) / pow(Rt, 1.0 / n) * pow(num / den, 1.0 / (2.0 * n));",
     "  return pow(eps_t, Rt) / pow(Rt, 1.0 / n) * pow(num / den, 1.0 / (2.0 * n));"),
    ("threshold_outer_power",
     "  return pow(eps_t, 1.0 / Rt) / pow(Rt, 1.0 / n) * pow(num / den, 1.0 / (2.0 * n));",
     "  return pow(eps_t, 1.0 / Rt) / pow(Rt, 1.0 / n) * pow(num / den, 1.0 / n);"),
    ("threshold_den_power",
     "  const double den = pow(eps_c, 2.0 * n / Rt) - pow(eps_t, 2.0 * n / Rt);",
     "  const double den = pow(eps_c, 2.0 * n * Rt) - pow(eps_t, 2.0 * n * Rt);"),
    # the mixture rule and sound speed (pins_sources.py)
    ("sound_speed_without_inverse_gamma",
     "    s += (arho[l] / ax->rho) * (1.0 / Gam) * cl2;",
     "    s += (arho[l] / ax->rho) * cl2;"),
    ("sound_speed_volume_weights",
     "    s += (arho[l] / ax->rho) * (1.0 / Gam) * cl2;",
     "    s += phi[l] * (1.0 / Gam) * cl2;"),
    ("sound_speed_without_dgamma",
     "    const double cl2 = mx->th[l][2] + (Gam + 1.0 + mx->th[l][5]) * (ax->p - mx->th[l][1]) /",
     "    const double cl2 = mx->th[l][2] + (Gam + 1.0) * (ax->p - mx->th[l][1]) /"),
    ("mixture_xi_times_gamma",
     "    mx->xi += phi[l] / mx->th[l][4];",
     "    mx->xi += phi[l] * mx->th[l][4];"),
    ("shear_speed_factor",
     "  const double cL2 = c2 + (4.0 / 3.0) * mx->Gmix / ax->rho;",
     "  const double cL2 = c2 + mx->Gmix / ax->rho;"),
    # the Riemann solver's wave and star speeds (pins_step.py)
    ("wave_speed_left_only",
     "  const double SL = a1 < a2 ? a1 : a2;",
     "  const double SL = a1;"),
    ("star_speed_traction_sign",
     "  const double Ss = (sL - sR + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /",
     "  const double Ss = (sR - sL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /"),
    ("star_side_swapped",
     "  star_side_flux(g, d, Ss >= 0.0, UL, aL, UR, aR, SL, SR, Ss, Fo, uface, Frow);",
     "  star_side_flux(g, d, Ss < 0.0, UL, aL, UR, aR, SL, SR, Ss, Fo, uface, Frow);"),
    # the sweep (pins_step.py, pins_waves.py)
    ("half_step_full_length",
     "      const double inc = 0.5 * lam * ((FL[k] - FR[k]) + nc[k]);",
     "      const double inc = lam * ((FL[k] - FR[k]) + nc[k]);"),
    ("limiter_not_harmonic",
     "  if (a * b > 0.0) return 2.0 * a * b / (a + b);",
     "  if (a * b > 0.0) return a * b / (a + b);"),
    ("slope_sign_left_face",
     "    wL[k] = wc[k] - 0.5 * s;",
     "    wL[k] = wc[k] + 0.5 * s;"),
    ("fbar_advection_sign",
     "    nc[g->o_F + c] = (2.0 / 3.0) * ac->F[3 * i + j] * du - ac->u[i] * dFrow[j];",
     "    nc[g->o_F + c] = (2.0 / 3.0) * ac->F[3 * i + j] * du + ac->u[i] * dFrow[j];"),
    ("phi_noncons_sign",
     "  for (int l = 0; l + 1 < g->nmat; ++l) nc[g->o_phi + l] = wc[g->o_phi + l] * du;",
     "  for (int l = 0; l + 1 < g->nmat; ++l) nc[g->o_phi + l] = -wc[g->o_phi + l] * du;"),
    ("X_noncons_dropped",
     "  for (int k = 0; k < g->dim; ++k) nc[g->o_X + k] = wc[g->o_X + k] * du;",
     "  for (int k = 0; k < g->dim; ++k) nc[g->o_X + k] = 0.0;"),
    ("update_noncons_sign",
     "          uc[k] + lam * ((FXr[(e - 1) * nf + k] - FX[e * nf + k]) + nc[k]);",
     "          uc[k] + lam * ((FXr[(e - 1) * nf + k] - FX[e * nf + k]) - nc[k]);"),
    ("cfl_without_sound_speed",
     "    v += ax.cL;",
     "    v += 0.0 * ax.cL + 1.0;"),
    ("weno3_weights_swapped",
     "  const double a1 = (2.0 / 3.0) / (e1 * e1);",
     "  const double a1 = (1.0 / 3.0) / (e1 * e1);"),
    ("void_stress_not_scaled",
     "const double pm = g->void_l >= 0 ? ax->p * (1.0 - phi[g->void_l]) : ax->p;",
     "const double pm = ax->p;"),
]


def _build(name, old, new, tmp):
    src = open(O.SRC).read()
    assert src.count(old) == 1, f"{name}: pattern occurs {src.count(old)} times"
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    return O.compile_oracle(path, os.path.join(tmp, f"lib{name}.so"))


# mistakes in the sweep are looked for first by the whole-step checks
STEP_FIRST = {"half_step_full_length", "limiter_not_harmonic", "slope_sign_left_face",
              "phi_noncons_sign", "X_noncons_dropped", "update_noncons_sign",
              "weno3_weights_swapped", "wave_speed_left_only", "star_speed_traction_sign",
              "star_side_swapped", "momentum_flux_stress_sign", "energy_flux_stress_row",
              "fbar_flux_row", "history_not_advected", "cfl_largest_spacing",
              "phase_bound_factor_two", "rk3_second_stage_weights", "rk3_last_stage_from_X1",
              "weno3_left_candidate"}


def _check(name, lib):
    # the closure, return, damage and lookup checks first (a second), the
    # fragment checks (a second or two), the void checks (a second or so),
    # the shear, wall, 3D and totals checks,
    # then the whole-step checks (ten seconds), which go first for a mistake
    # in the sweep
    mods = ["pins_sources.py", "pins_fragments.py", "pins_void.py", "pins_waves.py",
            "pins_step.py"]
    if name in STEP_FIRST:
        mods = ["pins_step.py"] + [m for m in mods if m != "pins_step.py"]
    out = ""
    for mod in mods:
        r = subprocess.run([sys.executable, os.path.join(HERE, mod), lib, "all"],
                           capture_output=True, text=True, timeout=900,
                           env=dict(os.environ, OMP_NUM_THREADS="2"))
        out = (r.stdout + r.stderr)[-400:]
        if r.returncode != 0:
            return r.returncode, out
    return 0, out


@functools.lru_cache(maxsize=None)
def _results():
    """Every copy built and checked once, in parallel (the unchanged copy,
    which runs every check, first)."""
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")
    jobs = [("unchanged", "#include <float.h>", "#include <float.h>")] + MUTANTS

    def run(job):
        name, old, new = job
        return name, _check(name, _build(name, old, new, tmp))

    try:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            return dict(ex.map(run, jobs))
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def test_every_planted_mistake_is_caught():
    res = {k: v for k, v in _results().items() if k != "unchanged"}
    assert len(res) == len(MUTANTS)
    survived = {k: v[1] for k, v in res.items() if v[0] == 0}
    assert not survived, f"mistakes no pin catches: {survived}"
    for k, (rc, out) in res.items():
        print(k, rc, out.strip().splitlines()[-1] if out.strip() else "")


def test_unplanted_copy_passes():
    # the same build route with nothing changed passes every check
    rc, out = _results()["unchanged"]
    assert rc == 0, out
