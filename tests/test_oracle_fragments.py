"""Pins of the oracle's fragment labelling (Sec. 4.2, 4.3: fragments are the
pieces demarcated by a void-fraction contour; in this gas-filled model a cell
is in a fragment when its solid fraction exceeds 1 - theta and no solid in it
is critically damaged).  Against scipy.ndimage.label on seeded random masks,
closed-form counts of cracked rings and cylinders, periodic joining, masses
summed independently, and the degenerate cases.  CPU only."""
import numpy as np
import pytest
from scipy import ndimage

import cases
from oracle import OracleGrid
from paper_2210_04037_gb300 import workloads as W


def members_from_prim(case, theta):
    """Membership written out from the primitive fields the case was made
    from (solid = material 0; critical = D >= D_crit within 1e-4)."""
    lay = case.layout
    phi = case.prim[lay.o_phi]
    Dc = case.materials[0]["D_crit"]
    crit = case.prim[lay.o_hist + 1] >= Dc * (1.0 - 1e-4)
    return (phi > 1.0 - theta) & ~crit


def random_mask_case(n, dim, seed, bc=W.BC_TRANSMISSIVE):
    """A ring or cylinder case whose solid fraction and damage are replaced
    by seeded per-cell draws: solid 0.2 or 0.8, a fifth of the cells
    critically damaged."""
    if dim == 2:
        case = W.ring_2d(n, seed=seed)
    else:
        case = W.cylinder_3d(n, nz=n, seed=seed)
    case.bc = [bc] * (2 * dim)
    lay = case.layout
    u = W.uniform01(seed + 100, 2 * case.ncell)
    case.prim[lay.o_phi] = np.where(u[: case.ncell] < 0.55, 0.8, 0.2)
    Dc = case.materials[0]["D_crit"]
    case.prim[lay.o_hist + 1] = np.where(u[case.ncell:] < 0.2, Dc, 0.5 * Dc)
    return case


def canonical(labels_scipy):
    """Relabel scipy's components by their smallest flat index (-1 outside)."""
    flat = labels_scipy.reshape(-1)
    out = np.full(flat.shape, -1, dtype=np.int64)
    for k in range(1, flat.max() + 1):
        idx = np.nonzero(flat == k)[0]
        out[idx] = idx.min()
    return out


@pytest.mark.parametrize("dim,n,seed", [(2, 40, 1), (2, 33, 2), (3, 14, 3), (3, 11, 4)])
@pytest.mark.parametrize("theta", [0.25, 0.5, 0.75])
def test_labels_match_scipy_on_random_masks(dim, n, seed, theta):
    case = random_mask_case(n, dim, seed)
    lab, f = OracleGrid(case).fragments(theta)
    mask = members_from_prim(case, theta)
    shape = tuple(case.n[:dim])[::-1]  # x fastest: arrays are (z, y, x)
    ref, nref = ndimage.label(mask.reshape(shape))  # face connectivity
    assert f["n"] == nref
    assert np.array_equal(lab, canonical(ref))
    assert np.array_equal(f["label"], np.unique(lab[lab >= 0]))
    assert np.array_equal(f["cells"], np.bincount(ref.reshape(-1))[1:][np.argsort(
        [np.nonzero(ref.reshape(-1) == k)[0].min() for k in range(1, nref + 1)])])


def test_periodic_faces_join_fragments():
    # a solid bar along x through the periodic faces: one fragment with
    # periodic x, two without
    for bc, expect in ((W.BC_PERIODIC, 1), (W.BC_TRANSMISSIVE, 2)):
        case = W.ring_2d(24)
        case.bc = [bc, bc, W.BC_TRANSMISSIVE, W.BC_TRANSMISSIVE]
        lay = case.layout
        x, y = case.centres()
        i = np.rint((x - case.lo[0]) / case.dx[0] - 0.5).astype(int)
        j = np.rint((y - case.lo[1]) / case.dx[1] - 0.5).astype(int)
        bar = (j >= 10) & (j < 13) & ((i < 5) | (i >= 19))
        case.prim[lay.o_phi] = np.where(bar, 1.0 - W.PHI_MIN, W.PHI_MIN)
        case.prim[lay.o_hist + 1] = 0.0
        lab, f = OracleGrid(case).fragments(0.5)
        assert f["n"] == expect
        assert f["cells"].sum() == bar.sum()
        assert f["label"][0] == int(np.nonzero(bar)[0].min())


@pytest.mark.parametrize("theta", [0.25, 0.5, 0.75])
def test_cracked_ring_falls_into_one_fragment_per_crack(theta):
    for k in (2, 5, 12):
        lab, f = OracleGrid(W.fractured_ring(160, cracks=k, seed=20 + k)).fragments(theta)
        assert f["n"] == k


def test_cracked_cylinder_falls_into_patches():
    # 8 axial cracks x 3 circumferential cracks on a z-periodic shell: 24
    # patches; one circumferential crack away from the ends: 8 with z
    # periodic (the tube opens once), 16 with z transmissive
    lab, f = OracleGrid(W.fractured_cylinder(64, 8, 3, nz=40)).fragments(0.5)
    assert f["n"] == 24
    case = W.fractured_cylinder(64, 8, 0, nz=40)
    lay = case.layout
    z = case.centres()[2]
    k = np.rint((z - case.lo[2]) / case.dx[2] - 0.5).astype(int)
    Dc = case.materials[0]["D_crit"]
    case.prim[lay.o_hist + 1] = np.where(k == 17, Dc, case.prim[lay.o_hist + 1])
    assert OracleGrid(case).fragments(0.5)[1]["n"] == 8
    case.bc = list(case.bc[:4]) + [W.BC_TRANSMISSIVE] * 2
    assert OracleGrid(case).fragments(0.5)[1]["n"] == 16


def test_masses_are_the_members_solid_mass_and_nest_in_theta():
    case = W.fractured_ring(128, cracks=7, seed=5)
    lay = case.layout
    dV = case.dx[0] * case.dx[1]
    arho = case.prim[lay.o_phi] * case.prim[lay.o_rho]  # solid phi rho from the inputs
    o = OracleGrid(case)
    prev_mask, prev_mass = None, 0.0
    for theta in (0.25, 0.5, 0.75):
        lab, f = o.fragments(theta)
        mask = lab >= 0
        assert np.array_equal(mask, members_from_prim(case, theta))
        for L, m in zip(f["label"], f["mass"]):
            assert m == pytest.approx(arho[lab == L].sum() * dV, rel=1e-12)
        if prev_mask is not None:
            assert np.all(mask[prev_mask])  # members at a lower cut-off stay members
            assert f["mass"].sum() > prev_mass
        prev_mask, prev_mass = mask, f["mass"].sum()


def test_degenerate_states():
    gas = OracleGrid(cases.gas_riemann(50, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)))
    lab, f = gas.fragments(0.5)
    assert f["n"] == 0 and np.all(lab == -1)
    bar = cases.elastic_cube(64, 0.01, lambda x: np.zeros_like(x))
    o = OracleGrid(bar)
    lab, f = o.fragments(0.5)
    assert f["n"] == 1 and f["cells"][0] == 64 and np.all(lab == 0)
    assert f["mass"][0] == pytest.approx(o.totals()[0], rel=1e-13)
    # max_frag smaller than the count: the count stays, the list is cut
    lab, f = OracleGrid(W.fractured_ring(96, cracks=6, seed=3)).fragments(0.5, max_frag=2)
    assert f["n"] == 6 and len(f["label"]) == 2
