"""The seeded input generators lay out what their docstrings state: the
fractured shells' solid fractions stay clear of the fragment cut-offs (so
the FP32 and FP64 membership decisions cannot differ), their cracks carry
D = D_crit and the rest D <= 0.9 D_crit, and the same seed gives the same
state.  CPU only; no arithmetic of the method."""
import numpy as np
import pytest

from paper_2210_04037_gb300 import workloads as W

CUTS = (0.25, 0.5, 0.75)


@pytest.mark.parametrize("make", [lambda: W.fractured_ring(128, cracks=9, seed=4),
                                  lambda: W.fractured_cylinder(48, 6, 2, nz=30, seed=5)])
def test_fractured_inputs(make):
    case = make()
    lay = case.layout
    phi = case.prim[lay.o_phi]
    for c in CUTS:
        assert np.min(np.abs(phi - (1.0 - c))) > 1e-3
    Dc = case.materials[0]["D_crit"]
    D = case.prim[lay.o_hist + 1]
    crack = D == Dc
    assert crack.any() and np.all(D[~crack] <= 0.9 * Dc)
    again = make()
    assert np.array_equal(case.prim, again.prim)
