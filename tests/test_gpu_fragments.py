"""Fragment labelling on the GPU (mm_fragments) against the oracle on seeded
fractured rings and z-periodic cylinder shells: labels and cell counts bit
for bit, masses to the summation bound (FP64 state: n_cells * 2^-52
relative; FP32-split state, whose phi rho is stored in FP32: 1e-6), at
three cut-offs, ragged sizes and the full bench sizes; the degenerate cases;
and, after steps on the GPU, the properties every labelling has."""
import numpy as np
import pytest

import cases
from oracle import OracleGrid
from paper_2210_04037_gb300 import mmfrac, workloads as W

pytestmark = pytest.mark.gpu

PRECS = [mmfrac.FP64, mmfrac.FP32_SPLIT]


def check_parity(case, prec, thetas=(0.25, 0.5, 0.75)):
    g = mmfrac.Grid(case, prec)
    o = OracleGrid(case)
    for theta in thetas:
        lab, f = g.fragments(theta)
        olab, of = o.fragments(theta)
        assert f["n"] == of["n"], theta
        assert np.array_equal(lab, olab), theta
        assert np.array_equal(f["label"], of["label"])
        assert np.array_equal(f["cells"], of["cells"])
        tol = of["cells"] * 2.0 ** -52 if prec == mmfrac.FP64 else 1e-6
        assert np.all(np.abs(f["mass"] - of["mass"]) <= tol * of["mass"]), theta
    g.close()
    return f["n"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,k", [(160, 5), (250, 12), (97, 3)])
def test_fractured_ring_matches_oracle(prec, n, k):
    assert check_parity(W.fractured_ring(n, cracks=k, seed=30 + n), prec) == k


@pytest.mark.parametrize("prec", PRECS)
def test_fractured_cylinder_matches_oracle(prec):
    # 8 x 3 patches across the z-periodic faces; then z transmissive
    case = W.fractured_cylinder(64, 8, 3, nz=40, seed=41)
    assert check_parity(case, prec) == 24
    case.bc = list(case.bc[:4]) + [W.BC_TRANSMISSIVE] * 2
    check_parity(case, prec, thetas=(0.5,))


@pytest.mark.parametrize("prec", PRECS)
def test_random_masks_match_oracle(prec):
    # many small fragments of every shape: seeded per-cell solid fraction and damage
    for dim, n, seed in ((2, 75, 7), (3, 23, 8)):
        case = W.ring_2d(n, seed=seed) if dim == 2 else W.cylinder_3d(n, nz=n - 3, seed=seed)
        lay = case.layout
        u = W.uniform01(seed + 100, 2 * case.ncell)
        case.prim[lay.o_phi] = np.where(u[: case.ncell] < 0.55, 0.8, 0.2)
        Dc = case.materials[0]["D_crit"]
        case.prim[lay.o_hist + 1] = np.where(u[case.ncell:] < 0.2, Dc, 0.5 * Dc)
        assert check_parity(case, prec) > 10


def test_full_size_ring_and_cylinder_match_oracle():
    # the bench sizes: 512^2 ring with 16 cracks, 256^3 shell with 12 x 4
    assert check_parity(W.fractured_ring(512, cracks=16, seed=5), mmfrac.FP32_SPLIT,
                        thetas=(0.5,)) == 16
    assert check_parity(W.fractured_cylinder(256, 12, 4, seed=6), mmfrac.FP32_SPLIT,
                        thetas=(0.5,)) == 48


def test_spall_1d_fragments():
    case = W.spall_1d(1000)
    lay = case.layout
    Dc = case.materials[0]["D_crit"]
    x = case.centres()[0]
    case.prim[lay.o_hist + 1] = np.where((np.abs(x - 0.0055) < 6e-5) | (np.abs(x - 0.0072) < 6e-5),
                                         Dc, 0.0)
    for prec in PRECS:
        assert check_parity(case, prec) == 3  # flyer and target in contact, cut twice


def test_degenerate_cases_and_arguments():
    g = mmfrac.Grid(cases.gas_riemann(64, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)), mmfrac.FP64)
    lab, f = g.fragments(0.5)
    assert f["n"] == 0 and np.all(lab == -1) and len(f["label"]) == 0
    g.close()
    case = cases.elastic_cube(100, 0.01, lambda x: np.zeros_like(x))
    g = mmfrac.Grid(case, mmfrac.FP32_SPLIT)
    lab, f = g.fragments(0.5)
    assert f["n"] == 1 and f["cells"][0] == 100 and np.all(lab == 0)
    assert f["mass"][0] == pytest.approx(g.totals()[0], rel=1e-6)
    g.close()
    g = mmfrac.Grid(W.fractured_ring(128, cracks=9, seed=2), mmfrac.FP32_SPLIT)
    lab, f = g.fragments(0.5, labels=False, max_frags=4)
    assert lab is None and f["n"] == 9 and len(f["label"]) == 4
    _, full = g.fragments(0.5)
    assert np.array_equal(f["label"], full["label"][:4])
    for bad in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(mmfrac.MMError) as e:
            g.fragments(bad)
        assert e.value.status == mmfrac.MM_EINVAL
    g.close()


@pytest.mark.parametrize("prec", PRECS)
def test_labels_after_steps_are_a_valid_labelling(prec):
    # after GPU steps the oracle has no copy of the state: check the
    # properties that define the labelling instead
    case = W.fractured_ring(200, cracks=7, seed=9)
    g = mmfrac.Grid(case, prec)
    g.step(25)
    lab, f = g.fragments(0.5)
    n = case.n[0]
    L = lab.reshape(n, n)
    for a, b in ((L[:, :-1], L[:, 1:]), (L[:-1, :], L[1:, :])):
        both = (a >= 0) & (b >= 0)
        assert np.array_equal(a[both], b[both])  # face neighbours share labels
    idx = np.nonzero(lab >= 0)[0]
    assert np.all(lab[idx] <= idx) and np.all(lab[lab[idx]] == lab[idx])
    assert np.array_equal(np.unique(lab[idx]), f["label"])
    assert np.array_equal(np.bincount(np.searchsorted(f["label"], lab[idx])), f["cells"])
    cons = g.read(False)
    dV = case.dx[0] * case.dx[1]
    arho = cons[case.layout.o_rho]
    sums = np.bincount(np.searchsorted(f["label"], lab[idx]), weights=arho[idx] * dV)
    assert np.allclose(f["mass"], sums, rtol=1e-9)
    # the 1.5-cell cracks heal within these steps: advection mixes their
    # D = D_crit with the undamaged neighbours (the healing Sec. 3.1 names)
    assert f["n"] >= 1
    g.close()


def test_labels_are_the_same_on_every_call():
    # the labelling's result does not depend on the order in which the
    # threads' unions and root stores land
    case = W.fractured_ring(512, cracks=16, seed=12)
    g = mmfrac.Grid(case, mmfrac.FP32_SPLIT)
    ref, _ = OracleGrid(case).fragments(0.5)
    for _ in range(6):
        lab, f = g.fragments(0.5)
        assert np.array_equal(lab, ref)
    g.close()
