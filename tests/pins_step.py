"""The whole-step pins of tests/test_oracle_pins.py (Toro's tests, Sod,
uniform state, contact equilibrium, conservation, mirror symmetry, elastic
and plastic wave fronts, second-order convergence, the WENO3 + RK3 X
transport and the half step's phase-density bound), run against a given
oracle library, so that copies of the oracle with a planted mistake in the
sweep can be checked too (tests/test_oracle_mutants.py).  No GPU.

Run as a script (``python pins_step.py LIB all``) it exits 0 when every
check passes against the library at LIB ("-": the oracle as built) and 1 at
the first failure."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import test_oracle_pins as T  # noqa: E402

CHECKS = {
    "cfl_sound_speeds": T.test_longitudinal_sound_speed_of_cube_and_air,
    "uniform_state": T.test_uniform_state_is_preserved_bitwise,
    "equilibrium_two_gases": T.test_interface_equilibrium_two_gases_exact,
    "equilibrium_copper_in_gas": T.test_interface_equilibrium_copper_in_gas,
    "conservation": T.test_conservation_on_periodic_box,
    "mirror": T.test_mirror_symmetry,
    "anisotropic_time_step": T.test_time_step_is_stable_on_an_anisotropic_grid,
    "elastic_wave_speed": T.test_elastic_wave_speed_in_cube,
    "elastic_precursor": T.test_elastic_precursor_of_plastic_impact,
    "second_order": T.test_second_order_convergence_on_smooth_elastic_wave,
    "sod": T.test_sod_error_at_1000_cells,
    "toro": lambda: [T.test_gas_limit_converges_to_exact_riemann_solution(k) for k in range(5)],
    "weno3_linear_X": lambda: [T.test_weno3_rk3_transports_a_linear_X_exactly(d, v)
                               for d, v in ((1, (100.0,)), (1, (-70.0,)), (2, (80.0, -50.0)))],
    "weno3_third_order": lambda: [T.test_weno3_rk3_X_transport_is_third_order(u)
                                  for u in (100.0, -100.0)],
    "weno3_only_X": T.test_weno3_rk3_X_is_the_only_field_that_changes_scheme,
    "half_step_bound_idle": lambda: [T.test_half_step_bound_leaves_physical_compression_alone(n, c)
                                     for n in T.PHYSICAL for c in (0.9, 1.0)],
    "half_step_bound_acts": T.test_half_step_bound_acts_on_trace_fractions_and_runs_stay_admissible,
}


if __name__ == "__main__":
    from oracle import oracle as _o
    if sys.argv[1] != "-":
        # every load() of the checks (and every OracleGrid they build) now
        # takes this copy
        _o._lib = _o.load_from(sys.argv[1])
    names = list(CHECKS) if sys.argv[2] == "all" else [sys.argv[2]]
    for name in names:
        try:
            CHECKS[name]()
        except Exception as e:  # a wrong value, or a copy that stops with an error code
            print(f"{name}: fails: {type(e).__name__}: {str(e)[:200]}")
            sys.exit(1)
    print("passes: " + " ".join(names))
    sys.exit(0)
