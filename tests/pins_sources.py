"""The closure (with the mixture rule and sound speed), Hencky-strain,
plastic-return, damage and perturbation-lookup pins of
tests/test_oracle_pins.py, run against a given oracle library, so
that copies of the oracle with a planted mistake in those parts can be
checked too (tests/test_oracle_mutants.py).  No GPU.

Run as a script (``python pins_sources.py LIB all``) it exits 0 when every
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
    "hencky": T.test_hencky_matches_matrix_logarithm,
    "cold_pressure": T.test_cold_pressure_is_density_derivative_of_cold_energy,
    "moduli": T.test_linear_moduli_at_reference_density,
    "steinberg": T.test_steinberg_closure_at_reference_and_its_grueneisen_derivative,
    "steinberg_sound_speed": T.test_steinberg_sound_speed_is_isentropic_derivative,
    "mixture_rule": T.test_ideal_gas_mixture_pressure_is_textbook_rule,
    "mixture_sound_speed": T.test_mixture_sound_speed_is_isentropic_derivative,
    "return_on_yield_surface": lambda: [
        T.test_perfectly_plastic_return_lands_on_perturbed_yield_surface(ph, Dm)
        for ph, Dm in ((1.0, 0.0), (1.13, 0.0), (0.87, 0.3))],
    "return_elastic_and_critical": T.test_elastic_state_is_unchanged_and_critical_damage_removes_strength,
    "return_rate_dependent": T.test_rate_dependent_return_satisfies_yield_condition,
    "unimodular": T.test_source_step_makes_fbar_unimodular,
    "damage_simple": T.test_simple_damage_matches_closed_form,
    "damage_bonora": T.test_bonora_damage_matches_closed_form_at_unit_triaxiality,
    "threshold_at_unit_triaxiality": T.test_threshold_strain_reduces_to_eps_thresh_at_unit_triaxiality,
    "threshold_limit": T.test_threshold_strain_in_the_limit_of_equal_strains,
    "triaxiality_forms": T.test_triaxiality_forms_agree_under_log_eos,
    "lookup": lambda: [T.test_lookup_is_multilinear(d) for d in (1, 2, 3)],
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
