"""The seeded input generators lay out what their docstrings state: the
random streams have the distributions they name (uniform, standard normal,
the rectified-normal and uniform perturbation fields), the fractured
shells' solid fractions stay clear of the fragment cut-offs (so the FP32 and
FP64 membership decisions cannot differ), their cracks carry D = D_crit and
the rest D <= 0.9 D_crit, and the same seed gives the same state.  CPU only;
no arithmetic of the method."""
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


def test_uniform_stream_is_uniform_and_offsets_agree():
    """53-bit uniforms in [0, 1) (reading R24): a Kolmogorov-Smirnov test
    against U(0, 1) on 2e5 draws, mean and variance within five standard
    errors; a stream read from an offset equals the tail of the whole."""
    from scipy import stats
    u = W.uniform01(11, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    assert np.array_equal(W.uniform01(11, 1000, start=500), W.uniform01(11, 1500)[500:])
    assert len(np.unique(W.splitmix64(11, 100_000))) == 100_000
    assert not np.array_equal(W.uniform01(11, 100), W.uniform01(12, 100))


def test_gaussian_draws_are_standard_normal():
    """Box-Muller on consecutive uniform pairs (R24): a Kolmogorov-Smirnov
    test against N(0, 1) on 1e5 draws, mean and standard deviation within
    five standard errors."""
    from scipy import stats
    g = W.gaussian(5, 100_000)
    assert np.all(np.isfinite(g))
    assert stats.kstest(g, "norm").pvalue > 1e-4
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    assert abs(g.std() - 1.0) < 5 / np.sqrt(2 * g.size)


def test_perturbation_fields_have_the_stated_distributions():
    """phi0 ~ rectified N(1, sd^2) (negative draws set to 0) and
    phi0 ~ U(1 - a, 1 + a) (Sec. 3.2.2; a uniform field with standard
    deviation s takes a = s sqrt(3), reading R21)."""
    gsd = W.perturbation_gaussian(3, (50, 40, 30), 0.1)
    assert gsd.dtype == np.float32 and gsd.size == 60_000
    assert abs(gsd.mean() - 1.0) < 5 * 0.1 / np.sqrt(gsd.size)
    assert abs(gsd.std() - 0.1) < 5 * 0.1 / np.sqrt(2 * gsd.size)
    wide = W.perturbation_gaussian(3, (60_000,), 1.0)
    assert wide.min() == 0.0 and np.mean(wide == 0.0) == pytest.approx(0.1587, abs=0.01)
    a = 0.2 * np.sqrt(3.0)
    uni = W.perturbation_uniform(4, (60_000,), a)
    assert uni.min() >= np.float32(1 - a) and uni.max() <= np.float32(1 + a)
    assert abs(uni.std() - 0.2) < 5 * 0.2 / np.sqrt(uni.size)
