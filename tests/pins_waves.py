"""Pins of the oracle's shear-wave branch, boundary rules, 3D sweeps and
totals against closed forms and symmetries (no GPU).  Each check takes the
oracle library as an argument (None: the oracle as built) so that the same
checks also run against copies of the oracle with a planted mistake
(tests/test_oracle_mutants.py), where at least one of them must fail.

Run as a script (``python pins_waves.py LIB CHECK``) it exits 0 when CHECK
passes against the library at LIB and 1 when an assertion fails."""
import os
import sys

import numpy as np
import scipy.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import cases  # noqa: E402
from oracle import OracleGrid  # noqa: E402
from paper_2210_04037_gb300 import workloads as W  # noqa: E402

CUBE = W.cube(damage="none", plastic=False)
AL = W.al_h32(damage="none", plastic=False)


def shear_speed(m):
    return np.sqrt(m["G0"] / m["rho0"])


def run_to(g, tend):
    t = 0.0
    while t < tend * (1 - 1e-14):
        dt, _ = g.cfl_dt()
        dt = min(dt, tend - t)
        g.step(1, dt=dt)
        t += dt


def sigma_xy(case, w, G):
    """Shear stress 2 G dev(H)_xy of each cell from its primitive Fbar
    (H = 1/2 ln(Fbar Fbar^T), by scipy), G the cells' shear modulus."""
    lay = case.layout
    out = np.empty(case.ncell)
    for c in range(case.ncell):
        F = np.eye(3)
        for comp in W.F_COMPS[case.dim]:
            i, j = divmod(comp, 3)
            F[i, j] = w[lay.F_index(i, j), c]
        H = 0.5 * np.real(sla.logm(F @ F.T))
        H -= np.trace(H) / 3 * np.eye(3)
        out[c] = 2 * G[c] * H[0, 1]
    return out


# --------------------------------------------------------------------------
# shear waves (the elastic system of Sec. 2.1 with the HLLD-type solver)
# --------------------------------------------------------------------------

def check_transverse_pulse_speed(lib=None):
    """A small transverse velocity pulse u_y(x) in CuBe splits into two
    shear waves travelling at sqrt(G0/rho0) (about 2531 m/s), the
    small-strain elastic shear speed."""
    L = 4e-3
    c = cases.shear_bar_2d(800, L, lambda x: 1.0 * np.exp(-((x - L / 2) / 1e-4) ** 2))
    g = OracleGrid(c, lib=lib)
    cs = shear_speed(CUBE)
    tend = 0.25 * L / cs
    run_to(g, tend)
    w = g.read()
    x = c.centres()[0]
    uy = w[c.layout.o_u + 1]
    right = x > L / 2
    xr = np.sum(x[right] * uy[right]) / np.sum(uy[right])
    assert abs((xr - L / 2) / tend / cs - 1) < 5e-3, (xr - L / 2) / tend
    # the two halves carry half the pulse each, left and right alike
    assert abs(np.sum(uy[right]) / np.sum(uy[~right]) - 1) < 1e-10


def shear_riemann(n, vL, vR, left=None, right=None, lib=None, frac_t=0.3):
    """Shear Riemann problem: u_y = vL left of the middle, vR right of it,
    no normal motion; run to frac_t L / c_s,max."""
    L = 4e-3
    x0 = L / 2
    c = cases.shear_bar_2d(n, L, lambda x: np.where(x < x0, vL, vR), left=left, right=right,
                           x0=x0)
    mats = c.materials
    cmax = max(shear_speed(m) for m in mats)
    tend = frac_t * L / cmax
    g = OracleGrid(c, lib=lib)
    run_to(g, tend)
    return c, g.read(), tend


def check_shear_riemann_symmetric(lib=None):
    """u_y = -v | +v in CuBe.  The exact small-strain solution has a shear
    wave each way at c_s = sqrt(G0/rho0), between them u_y = 0 and the
    continuous traction sigma_xy = rho0 c_s v.  The problem is invariant
    under the mirror in x combined with the mirror in y, so the numerical
    solution has u_y(x) = -u_y(L - x) and sigma_xy(x) = sigma_xy(L - x) to
    rounding."""
    v = 10.0
    c, w, t = shear_riemann(400, -v, v)
    lay = c.layout
    x = c.centres()[0]
    row = slice(0, 400)  # the first of the two identical rows along y
    uy = w[lay.o_u + 1][row]
    assert np.abs(uy + uy[::-1]).max() <= 1e-12 * v
    cs = shear_speed(CUBE)
    G = np.full(c.ncell, CUBE["G0"]) * (w[lay.o_rho] / CUBE["rho0"]) ** (CUBE["beta"] + 1)
    sxy = sigma_xy(c, w, G)[row]
    assert np.abs(sxy - sxy[::-1]).max() <= 1e-9 * CUBE["rho0"] * cs * v
    xm = x[row]
    L = c.hi[0]
    plateau = np.abs(xm - L / 2) < 0.5 * cs * t
    assert np.abs(uy[plateau]).max() < 0.02 * v
    tau = CUBE["rho0"] * cs * v
    assert abs(np.median(sxy[plateau]) / tau - 1) < 0.01
    assert np.std(sxy[plateau]) < 0.01 * tau
    # fronts: u_y crosses +-v/2 at L/2 +- c_s t
    dx = c.dx[0]
    xr = xm[(xm > L / 2) & (uy > 0.5 * v)].min()
    xl = xm[(xm < L / 2) & (uy < -0.5 * v)].max()
    assert abs(xr - (L / 2 + cs * t)) < 2 * dx and abs(xl - (L / 2 - cs * t)) < 2 * dx


def check_shear_riemann_bimaterial(lib=None):
    """u_y = vL | vR across a CuBe / Al-H32 interface (volume fractions
    1 - 1e-6 / 1e-6).  Linear elasticity gives, between the left shear wave
    at -c_1 t and the right one at +c_2 t, the interface velocity
    u* = (Z1 vL + Z2 vR)/(Z1 + Z2) and the traction
    tau* = Z1 Z2 (vR - vL)/(Z1 + Z2) (Z = sqrt(rho G), the shear impedance):
    unequal impedances make the answer depend on which side each term of
    the solver takes."""
    vL, vR = -4.0, 12.0
    c, w, t = shear_riemann(600, vL, vR, left=CUBE, right=AL, lib=lib, frac_t=0.3)
    lay = c.layout
    n = c.n[0]
    x = c.centres()[0][:n]
    L = c.hi[0]
    Z1, Z2 = np.sqrt(CUBE["rho0"] * CUBE["G0"]), np.sqrt(AL["rho0"] * AL["G0"])
    c1, c2 = shear_speed(CUBE), shear_speed(AL)
    us = (Z1 * vL + Z2 * vR) / (Z1 + Z2)
    tau = Z1 * Z2 * (vR - vL) / (Z1 + Z2)
    phi = w[lay.o_phi]
    rho = np.stack([w[lay.o_rho], w[lay.o_rho + 1]])
    G = sum((phi if l == 0 else 1 - phi) * m["G0"] * (rho[l] / m["rho0"]) ** (m["beta"] + 1)
            for l, m in enumerate((CUBE, AL)))
    uy = w[lay.o_u + 1][:n]
    sxy = sigma_xy(c, w, G)[:n]
    dx = c.dx[0]
    for lo, hi in ((L / 2 - 0.75 * c1 * t, L / 2 - 4 * dx), (L / 2 + 4 * dx, L / 2 + 0.75 * c2 * t)):
        band = (x > lo) & (x < hi)
        assert band.sum() >= 10
        assert np.abs(uy[band] - us).max() < 0.01 * (vR - vL), (np.median(uy[band]), us)
        assert np.abs(sxy[band] / tau - 1).max() < 0.01, (np.median(sxy[band]), tau)
    xr = x[(x > L / 2) & (uy > 0.5 * (us + vR))].min()
    xl = x[(x < L / 2) & (uy < 0.5 * (us + vL))].max()
    assert abs(xr - (L / 2 + c2 * t)) < 2 * dx and abs(xl - (L / 2 - c1 * t)) < 2 * dx


def thermal_pressure(case, w, mats):
    """p - p_ref(rho_l, J2) of each cell of a shear bar: the part of the
    pressure carried by the thermal energy, from the pinned equation of
    state of the oracle as built (Romenskii reference curve with the shear
    term; the cell's majority material)."""
    import ctypes
    from oracle import load, material_struct
    lib0 = load()
    lay = case.layout
    out = np.empty(case.ncell)
    buf = np.zeros(6)
    pb = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    structs = [material_struct(m) for m in mats]
    for c in range(case.ncell):
        F = np.eye(3)
        for comp in W.F_COMPS[case.dim]:
            i, j = divmod(comp, 3)
            F[i, j] = w[lay.F_index(i, j), c]
        H = 0.5 * np.real(sla.logm(F @ F.T))
        H -= np.trace(H) / 3 * np.eye(3)
        l = 0 if len(mats) == 1 or w[lay.o_phi, c] > 0.5 else 1
        lib0.or_thermo(ctypes.byref(structs[l]), w[lay.o_rho + l, c], 1.0, float(np.sum(H * H)), pb)
        out[c] = w[lay.o_p, c] - buf[1]
    return out


def check_shear_waves_do_not_cool(lib=None):
    """Shear waves are isentropic and numerical dissipation only heats: in
    the symmetric and the bimaterial shear Riemann problems the thermal
    part of the pressure (p less the reference-curve pressure at the cell's
    density and shear invariant) stays at or above its initial 1e5 Pa
    between the interface and the shear fronts."""
    for args, mats in (((400, -10.0, 10.0), [CUBE]),
                       ((600, -4.0, 12.0, CUBE, AL), [CUBE, AL])):
        c, w, t = shear_riemann(*args, lib=lib)
        n = c.n[0]
        x = c.centres()[0][:n]
        L, dx = c.hi[0], c.dx[0]
        pth = thermal_pressure(c, w, mats)[:n]
        for lo, hi in ((L / 2 - 0.75 * shear_speed(mats[0]) * t, L / 2 - 4 * dx),
                       (L / 2 + 4 * dx, L / 2 + 0.75 * shear_speed(mats[-1]) * t)):
            band = (x > lo) & (x < hi)
            assert pth[band].min() >= 1e5 * (1 - 1e-3), (len(mats), pth[band].min())


def check_shear_tangential_galilean(lib=None):
    """The bimaterial shear Riemann problem boosted by 50 m/s along y: the
    same solution with u_y shifted by 50 m/s (and X_y by 50 t): the star
    states of the solver carry the boost in every term, on either side."""
    U = 50.0
    L = 4e-3
    runs = []
    for v0 in (0.0, U):
        c0 = cases.shear_bar_2d(600, L, lambda x: np.where(x < L / 2, -4.0, 12.0) + v0,
                                left=CUBE, right=AL, x0=L / 2)
        g = OracleGrid(c0, lib=lib)
        # one fixed time step for both runs (the CFL step sees |u_y| and
        # would differ between them): 0.4 of the boosted run's CFL limit
        if not runs:
            dt = 0.4 * c0.dx[0] / (np.sqrt((CUBE["K0"] + 4 / 3 * CUBE["G0"]) / CUBE["rho0"]) + 62.0)
        g.step(int(0.3 * L / shear_speed(AL) / dt), dt=dt)
        runs.append(g.read())
    w0, w1 = runs
    lay = c0.layout
    for f in range(lay.nfield):
        if f == lay.o_X + 1:
            continue
        ref = w0[f] + (U if f == lay.o_u + 1 else 0.0)
        # velocities on the scale of the shear jump (16 m/s)
        scale = 16.0 if lay.o_u <= f < lay.o_u + 2 else np.abs(ref).max() + 1e-300
        err = np.abs(w1[f] - ref).max() / scale
        assert err <= 1e-8, (lay.names()[f], err)


# --------------------------------------------------------------------------
# boundary rules: a reflective box is half of a mirrored, doubled periodic box
# --------------------------------------------------------------------------

def reflective_case(kind):
    if kind == "gas_1d":
        c = cases.gas_riemann(120, (1.0, 0.75, 1.0), (0.125, -0.4, 0.1), x0=0.37)
        c.bc = [W.BC_REFLECTIVE] * 2
        return c, 0, 60
    if kind == "solid_1d":
        c = cases.spall_like_1d(160, v=400.0)
        c.bc = [W.BC_REFLECTIVE] * 2
        return c, 0, 120
    if kind == "mix_2d_x":
        c = cases.periodic_mix_2d(20, seed=4, shear=0.03, bc=W.BC_PERIODIC)
        c.bc = [W.BC_REFLECTIVE, W.BC_REFLECTIVE, W.BC_PERIODIC, W.BC_PERIODIC]
        return c, 0, 40
    if kind == "mix_2d_y":
        c = cases.periodic_mix_2d(20, seed=4, shear=0.03, bc=W.BC_PERIODIC)
        c.bc = [W.BC_PERIODIC, W.BC_PERIODIC, W.BC_REFLECTIVE, W.BC_REFLECTIVE]
        return c, 1, 40
    if kind == "mix_3d_z":
        c = cases.periodic_mix_3d(8, nz=10, bc=W.BC_PERIODIC)
        c.bc = [W.BC_PERIODIC] * 4 + [W.BC_REFLECTIVE] * 2
        return c, 2, 25
    raise KeyError(kind)


REFLECTIVE_KINDS = ("gas_1d", "solid_1d", "mix_2d_x", "mix_2d_y", "mix_3d_z")


def check_reflective_walls(kind, lib=None):
    """Reflective walls at both ends of an axis (ghosts mirrored: u_d and
    the Fbar comps with exactly one index d negated, X_d reflected about the
    wall) give the same run as the first half of the box doubled by its
    mirror image and made periodic along that axis, which has the walls'
    symmetry planes built in.  Equal in every conserved field to rounding
    (1D: 1e-13 of each field's scale; 2D and 3D, where the two halves of the
    doubled box drift apart by rounding and the drift grows over the run:
    1e-11)."""
    c, axis, steps = reflective_case(kind)
    d = cases.doubled_periodic(c, axis)
    g1, g2 = OracleGrid(c, lib=lib), OracleGrid(d, lib=lib)
    g1.step(steps)
    g2.step(steps)
    a = g1.read(False)
    b = cases.first_half(d, g2.read(False), axis)
    scale = np.abs(a).max(axis=1) + 1e-300
    err = (np.abs(a - b).max(axis=1) / scale).max()
    assert err <= (1e-13 if c.dim == 1 else 1e-11), (kind, err)


def check_reflective_box_mirror(kind, lib=None):
    """A box with reflective walls at both ends of an axis, mirrored about
    its mid-plane along that axis, evolves into the mirror image of its own
    run: the two walls are treated alike (to rounding, 1e-11 of each
    field's scale).  At a wall the contact is at rest and its Riemann
    problem is its own mirror image; taking one side's star state there
    (either one, by the sign of a rounded zero) puts a flux of the
    tangential rows of Fbar through the wall of opposite sign at the two
    ends, which breaks the symmetry at the 1e-4 level within a few
    steps."""
    c, axis, steps = reflective_case(kind)
    g = OracleGrid(c, lib=lib)
    g.step(steps)
    r = g.read(False)
    m = cases.mirrored(c, axis)
    gm = OracleGrid(m, lib=lib)
    gm.step(steps)
    back = cases.mirror_fields(m, gm.read(False), axis, c.lo[axis] + c.hi[axis])
    scale = np.abs(r).max(axis=1) + 1e-300
    err = (np.abs(back - r).max(axis=1) / scale).max()
    assert err <= 1e-11, (kind, err)


# --------------------------------------------------------------------------
# 3D: axis permutations, mirrors, conservation
# --------------------------------------------------------------------------

def check_axis_permutation(lib=None):
    """One 1D problem (plastic impact in air) and one 2D problem (compressed
    copper/air mixture with shear) laid along every axis of a 3D grid (the
    other axes two cells wide, periodic, uniform): the transverse sweeps
    leave uniform data unchanged, so every layout gives the 1D / 2D
    answer, with u, Fbar and X permuted with the axes.  Rounding differs
    only where a sum of three terms is taken in another order."""
    c1 = cases.spall_like_1d(64, v=300.0)
    ref1 = OracleGrid(c1, lib=lib)
    ref1.step(40)
    r1 = ref1.read(False)
    c2 = cases.periodic_mix_2d(14, seed=3, shear=0.03)
    ref2 = OracleGrid(c2, lib=lib)
    ref2.step(20)
    r2 = ref2.read(False)
    # 2D problems keep the sweep order of their two axes (x before y)
    for case, ref, steps, perms in ((c1, r1, 40, [(0,), (1,), (2,)]),
                                    (c2, r2, 20, [(0, 1), (0, 2), (1, 2)])):
        for perm in perms:
            c3, full, src = cases.embed_3d(case, perm)
            g = OracleGrid(c3, lib=lib)
            g.step(steps)
            out = cases.unembed_3d(case, c3, full, g.read(False), src)
            scale = np.abs(ref).max(axis=1) + 1e-300
            err = (np.abs(out - ref).max(axis=1) / scale).max()
            assert err <= 1e-11, (case.name, perm, err)


def check_mirror_3d(lib=None):
    """The 3D mixture mirrored about the mid-plane along x, y or z evolves
    into the mirror image of its own run (transmissive ends)."""
    c = cases.periodic_mix_3d(8, nz=10, bc=W.BC_TRANSMISSIVE)
    g = OracleGrid(c, lib=lib)
    g.step(12)
    r = g.read(False)
    scale = np.abs(r).max(axis=1) + 1e-300
    for axis in range(3):
        m = cases.mirrored(c, axis)
        gm = OracleGrid(m, lib=lib)
        gm.step(12)
        back = cases.mirror_fields(m, gm.read(False), axis, c.lo[axis] + c.hi[axis])
        err = (np.abs(back - r).max(axis=1) / scale).max()
        assert err <= 1e-11, (axis, err)


def check_conservation_3d(lib=None):
    """Masses, momenta and total energy on a periodic 3D box over 100 steps
    with the plastic return active: conserved to rounding (every sweep is in
    flux form for these fields; the sources change none of them)."""
    c = cases.periodic_mix_3d(10, nz=8)
    g = OracleGrid(c, lib=lib)
    lay = c.layout
    T0 = g.totals()
    U0 = g.read(False)
    dV = np.prod(c.dx)
    mscale = np.abs(U0[lay.o_u:lay.o_u + 3]).sum() * dV
    g.step(100)
    T1 = g.totals()
    assert abs(T1[0] / T0[0] - 1) < 1e-13 and abs(T1[1] / T0[1] - 1) < 1e-13
    assert np.abs(T1[2:5] - T0[2:5]).max() < 1e-13 * mscale
    assert abs(T1[5] / T0[5] - 1) < 1e-13
    assert g.read(False)[lay.o_hist].max() > 0  # plastic flow happened


# --------------------------------------------------------------------------
# totals
# --------------------------------------------------------------------------

def check_totals_closed_form(lib=None):
    """Totals of a state made of two uniform halves on a box with unequal
    cell sizes along x, y and z: (a + b)/2 times the box volume for every
    conserved density (masses, momenta, total energy)."""
    mats = [W.cube(), W.air()]
    c = W.Case("halves", 3, [6, 4, 10], [0, 0, 0], [3e-3, 1e-3, 7e-3], [0] * 6, mats, None)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    x, y, z = c.centres()
    half = z < 3.5e-3
    W.fill_two_phase(c, np.where(half, 0.8, 0.3), 8370.0, 1.2, 1e5,
                     [np.where(half, 30.0, -10.0), np.where(half, 5.0, 7.0), np.where(half, 0, 2.0)])
    g = OracleGrid(c, lib=lib)
    U = g.read(False)
    V = 3e-3 * 1e-3 * 7e-3
    T = g.totals()
    fields = [lay.o_rho, lay.o_rho + 1, lay.o_u, lay.o_u + 1, lay.o_u + 2, lay.o_p]
    for q, f in enumerate(fields):
        a, b = U[f][half][0], U[f][~half][0]
        assert np.all(U[f][half] == a) and np.all(U[f][~half] == b)
        assert abs(T[q] - 0.5 * (a + b) * V) <= 1e-14 * abs(0.5 * (a + b) * V) + 1e-300, (q, T[q])


CHECKS = {
    "totals_closed_form": check_totals_closed_form,
    "axis_permutation": check_axis_permutation,
    "mirror_3d": check_mirror_3d,
    "conservation_3d": check_conservation_3d,
    "shear_riemann_symmetric": check_shear_riemann_symmetric,
    "shear_riemann_bimaterial": check_shear_riemann_bimaterial,
    "transverse_pulse_speed": check_transverse_pulse_speed,
    "shear_waves_do_not_cool": check_shear_waves_do_not_cool,
    "shear_tangential_galilean": check_shear_tangential_galilean,
}
for _k in REFLECTIVE_KINDS:
    CHECKS["reflective_" + _k] = (lambda k: lambda lib=None: check_reflective_walls(k, lib))(_k)
    CHECKS["reflective_mirror_" + _k] = (
        lambda k: lambda lib=None: check_reflective_box_mirror(k, lib))(_k)


if __name__ == "__main__":
    # python pins_waves.py LIB NAME|all: exit 1 at the first check that fails
    # (an assertion, or the oracle rejecting a step), 0 when all pass
    from oracle import oracle as _o
    lib = _o.load_from(sys.argv[1]) if sys.argv[1] != "-" else None
    names = list(CHECKS) if sys.argv[2] == "all" else [sys.argv[2]]
    for name in names:
        try:
            CHECKS[name](lib)
        except (AssertionError, RuntimeError, ValueError) as e:
            print(f"{name}: fails: {type(e).__name__}: {e}")
            sys.exit(1)
    print("passes: " + " ".join(names))
    sys.exit(0)
