"""The fragment-labelling pins of tests/test_oracle_fragments.py, run against
a given oracle library, so that copies of the oracle with a planted mistake
in the labelling can be checked too (tests/test_oracle_mutants.py).  No GPU.

Run as a script (``python pins_fragments.py LIB all``) it exits 0 when every
check passes against the library at LIB ("-": the oracle as built) and 1 at
the first failure."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import test_oracle_fragments as T  # noqa: E402

CHECKS = {
    "scipy_random_masks": lambda: [T.test_labels_match_scipy_on_random_masks(d, n, s, th)
                                   for d, n, s in ((2, 40, 1), (2, 33, 2), (3, 14, 3), (3, 11, 4))
                                   for th in (0.25, 0.5, 0.75)],
    "periodic_faces": T.test_periodic_faces_join_fragments,
    "cracked_ring": lambda: [T.test_cracked_ring_falls_into_one_fragment_per_crack(th)
                             for th in (0.25, 0.5, 0.75)],
    "cracked_cylinder": T.test_cracked_cylinder_falls_into_patches,
    "masses": T.test_masses_are_the_members_solid_mass_and_nest_in_theta,
    "degenerate": T.test_degenerate_states,
}


if __name__ == "__main__":
    from oracle import oracle as _o
    if sys.argv[1] != "-":
        # every OracleGrid the checks build now takes this copy
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
