"""Pins of the oracle's void volume fraction and void-opening flux modifier
(Sec. 2.1 nu equation; Sec. 3.1 fracture; reading R33) against closed forms
(no GPU).  Checks take the oracle library as an argument, as in
pins_waves.py, so that copies of the oracle with a planted mistake can be
checked too.

The setting: a CuBe bar of 400 cells, at rest, in uniform hydrostatic
tension sigma0 (a negative pressure), with a critically damaged cell in the
middle.  Its faces are critical and in tension, so the void opens on both
sides of it at once: each half meets a traction-free surface.  Linear 1D
strain elasticity then gives release waves running into the halves at
c_L = sqrt((K0 + 4/3 G0)/rho0), the material behind them stress-free and
moving away from the crack at v = sigma0/(rho0 c_L), and a void volume
growing as 2 v t (the damaged cell, released on both sides, stays put).

Run as a script (``python pins_void.py LIB all``) it exits 0 when every
check passes against the library at LIB and 1 at the first failure."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

from oracle import OracleGrid  # noqa: E402
from paper_2210_04037_gb300 import workloads as W  # noqa: E402

CUBE = W.cube("bonora")
CL = np.sqrt((CUBE["K0"] + 4 / 3 * CUBE["G0"]) / CUBE["rho0"])
L = 4e-3
N = 400
SIGMA0 = 2e8


def bar(p=-SIGMA0, crack=(N // 2,), with_void=True, u=lambda x: 0 * x, n=N):
    """The bar: [void, CuBe] (or CuBe alone), pressure p (negative:
    tension), velocity u(x), cells in `crack` at D = D_crit, transmissive
    ends."""
    mats = [W.void(), CUBE] if with_void else [CUBE]
    c = W.Case("bar", 1, [n, 1, 1], [0, 0, 0], [L, 1, 1], [0, 0], mats, None, cfl=0.6)
    lay = c.layout
    c.prim = W.blank_prim(lay, n)
    x = c.centres()[0]
    k = 1 if with_void else 0
    if with_void:
        c.prim[lay.o_phi] = 0.0
        c.prim[lay.o_rho] = 0.0
    c.prim[lay.o_rho + k] = CUBE["rho0"]
    c.prim[lay.o_u] = u(x)
    c.prim[lay.o_p] = p
    D = np.zeros(n)
    D[list(crack)] = CUBE["D_crit"]
    c.prim[lay.o_hist + 1] = D
    c.prim[lay.o_X] = x
    return c


def run_to(g, tend, dt=None):
    t = 0.0
    while t < tend * (1 - 1e-14):
        step = g.cfl_dt()[0] if dt is None else dt
        step = min(step, tend - t)
        g.step(1, dt=step)
        t += step


def sigma_xx(case, w):
    """Normal stress of each cell from its primitive fields:
    -(1 - nu) p + 2 G dev(H)_xx, G = phi (1 - D) G0 (rho/rho0)^(beta+1) for
    the CuBe, H = ln Fbar (diagonal in 1D)."""
    lay = case.layout
    nu = w[lay.o_phi]
    rho = w[lay.o_rho + 1]
    D = w[lay.o_hist + 1]
    G = (1 - nu) * (1 - D) * CUBE["G0"] * (rho / CUBE["rho0"]) ** (CUBE["beta"] + 1)
    h = [np.log(w[lay.F_index(i, i)]) for i in range(3)]
    dev = h[0] - (h[0] + h[1] + h[2]) / 3
    return -(1 - nu) * w[lay.o_p] + 2 * G * dev


def mass(case, U, sl):
    lay = case.layout
    return U[lay.o_rho:lay.o_rho + len(case.materials), sl].sum() * case.dx[0]


def check_release_from_a_crack(lib=None):
    """Release waves at c_L, stress-free material moving off at
    v = sigma0/(rho0 c_L) behind them, void volume 2 v t, masses of the two
    halves and of the damaged cell kept exactly, fractions summing to one."""
    c = bar()
    g = OracleGrid(c, lib=lib)
    lay = c.layout
    U0 = g.read(False)
    t = 0.3 * L / CL
    run_to(g, t)
    w, U = g.read(), g.read(False)
    x = c.centres()[0]
    dx = c.dx[0]
    v = SIGMA0 / (CUBE["rho0"] * CL)
    nu = w[lay.o_phi]
    assert nu.min() >= 0.0 and nu.max() <= 1.0
    assert np.all(U[lay.o_phi] <= 1.0)
    sig = sigma_xx(c, w)
    # release fronts: sigma crosses sigma0/2 at L/2 -+ c_L t
    mid = L / 2
    right = x > mid + 2 * dx
    left = x < mid - 2 * dx
    xr = x[right & (sig > 0.5 * SIGMA0)].min()
    xl = x[left & (sig > 0.5 * SIGMA0)].max()
    for front, target in ((xr, mid + CL * t), (xl, mid - CL * t)):
        assert abs(front - target) < 0.02 * CL * t + 2 * dx, (front, target)
    # behind them: stress-free, moving away at v
    band_r = (x > mid + 5 * dx) & (x < mid + 0.8 * CL * t)
    band_l = (x < mid - 5 * dx) & (x > mid - 0.8 * CL * t)
    assert band_r.sum() > 20 and band_l.sum() > 20
    assert np.abs(sig[band_r | band_l]).max() < 0.03 * SIGMA0
    assert np.abs(np.median(w[lay.o_u][band_r]) / v - 1) < 0.03
    assert np.abs(np.median(w[lay.o_u][band_l]) / v + 1) < 0.03
    # the void volume is the gap, 2 v t
    gap = nu.sum() * dx
    assert abs(gap / (2 * v * t) - 1) < 0.05, (gap, 2 * v * t)
    # nothing crosses an opened face: the halves keep their mass (the
    # release has not reached the bar's ends) to 1e-6 of it: the opened
    # surfaces are stress-free, so the tension test there flips on the sign
    # of a near-zero stress, and a face that takes the contact solver for a
    # step moves a trace across (the damaged cell between them, whose mass
    # is 1/200 of a half's, exchanges 4e-5 of its own this way)
    k = N // 2
    for sl in (slice(0, k), slice(k + 1, N)):
        m0, m1 = mass(c, U0, sl), mass(c, U, sl)
        assert abs(m1 / m0 - 1) < 1e-6, (sl, m0, m1)
    assert abs(mass(c, U, slice(0, N)) / mass(c, U0, slice(0, N)) - 1) < 1e-14


def _same_as_without_void(c_void, c_plain, steps, lib):
    a, b = OracleGrid(c_void, lib=lib), OracleGrid(c_plain, lib=lib)
    a.step(steps)
    b.step(steps)
    ua, ub = a.read(False), b.read(False)
    lay = c_void.layout
    assert np.all(ua[lay.o_phi] == 0.0)  # no void opened
    # the void's fraction and (zero) mass are the two extra fields
    keep = [f for f in range(lay.nfield) if f not in (lay.o_phi, lay.o_rho)]
    assert np.array_equal(ua[keep], ub), np.abs(ua[keep] - ub).max()


def check_no_opening_in_compression(lib=None):
    """A critically damaged cell in compression: the modifier does not act,
    and the run equals the same bar without a void material bit for bit."""
    _same_as_without_void(bar(p=+SIGMA0), bar(p=+SIGMA0, with_void=False), 80, lib)


def check_no_opening_without_critical_damage(lib=None):
    """Tension without critical damage (D = 0.99 D_crit): no void opens and
    the run equals the bar without a void material bit for bit."""
    c1, c2 = bar(crack=()), bar(crack=(), with_void=False)
    lay = c1.layout
    c1.prim[lay.o_hist + 1][N // 2] = 0.99 * CUBE["D_crit"]
    c2.prim[c2.layout.o_hist + 1][N // 2] = 0.99 * CUBE["D_crit"]
    _same_as_without_void(c1, c2, 80, lib)


def check_opening_at_capped_damage(lib=None):
    """A crack at D = D_crit (1 - 1e-5), as a capped D reads back after
    advection, is critical (R34): the void opens as at D = D_crit (opened
    volume within 1e-4 after 40 steps; the damaged cell's moduli differ by
    (1 - D) between the two)."""
    gaps = []
    for D in (CUBE["D_crit"], CUBE["D_crit"] * (1 - 1e-5)):
        c = bar()
        c.prim[c.layout.o_hist + 1][N // 2] = D
        g = OracleGrid(c, lib=lib)
        g.step(40)
        gaps.append(g.read()[c.layout.o_phi].sum())
    assert gaps[0] > 0.01 and abs(gaps[1] / gaps[0] - 1) < 1e-4, gaps


def porous_bar(nu=0.5, p=1e8):
    """The bar without a crack: CuBe at pressure p on the left half, the same
    CuBe with void fraction nu at p / (1 - nu) on the right half."""
    c = bar(p=p, crack=())
    lay = c.layout
    right = c.centres()[0] > L / 2
    c.prim[lay.o_phi] = np.where(right, nu, 0.0)
    c.prim[lay.o_p] = np.where(right, p / (1 - nu), p)
    return c


def check_porous_stress_equilibrium(lib=None):
    """The void carries no stress (R33: the mixture's pressure is (1 - nu) p):
    the CuBe at p = 1e8 Pa beside the same CuBe with void fraction 0.5 at
    p = 2e8 Pa, at rest and unsheared, has the same normal stress on both
    sides, so it stays at rest (|u| below 1e-9 of p / (rho0 c_L) after 50
    steps) and the porosity jump stays where it is."""
    c = porous_bar()
    lay = c.layout
    g = OracleGrid(c, lib=lib)
    g.step(50)
    w = g.read()
    assert np.abs(w[lay.o_u]).max() < 1e-9 * 1e8 / (CUBE["rho0"] * CL), np.abs(w[lay.o_u]).max()
    assert np.array_equal(w[lay.o_phi], c.prim[lay.o_phi])


def check_void_opening_mirror(lib=None):
    """An off-centre crack in a bar in tension with a smooth velocity
    perturbation, mirrored about the mid-plane, runs into the mirror image
    of its own run over 100 steps (1e-11 of each field's scale): the
    decisions of the void opening (critical damage, tension, the clamps of
    a void fraction a rounding below zero) take the same branch on both."""
    pert = lambda x: 5.0 * np.sin(2 * np.pi * x / L)
    c = bar(crack=(N // 2 + 37,), u=pert)
    m = bar(crack=(N - 1 - (N // 2 + 37),), u=lambda x: -pert(L - x))
    m.prim[m.layout.o_X] = c.centres()[0]
    g1, g2 = OracleGrid(c, lib=lib), OracleGrid(m, lib=lib)
    g1.step(100)
    g2.step(100)
    a, b = g1.read(False), g2.read(False)
    lay = c.layout
    back = b[:, ::-1].copy()
    back[lay.o_u] *= -1.0
    back[lay.o_X] = L - back[lay.o_X]
    scale = np.abs(a).max(axis=1) + 1e-300
    err = (np.abs(back - a).max(axis=1) / scale).max()
    assert err <= 1e-11, err
    assert a[lay.o_phi].max() > 1e-3  # the void did open


def check_void_opening_galilean(lib=None):
    """The same crack with the bar moving at 150 m/s (a fixed time step for
    both): the void volume the first step opens is the same as at rest
    (1e-3), although the gap then lies on one side of each opening face,
    not across it (the surfaces move at 150 -/+ v).  (Later steps differ:
    the intact material advected into the damaged cell heals it below
    D_crit, the artificial healing of Sec. 3.1.)"""
    dt = 0.5 * (L / N) / (CL + 150.0)
    gaps = []
    for U in (0.0, 150.0):
        c = bar(u=lambda x, U=U: 0 * x + U)
        g = OracleGrid(c, lib=lib)
        g.step(1, dt=dt)
        w = g.read()
        gaps.append(w[c.layout.o_phi].sum() * c.dx[0])
    assert gaps[0] > 0 and abs(gaps[1] / gaps[0] - 1) < 1e-3, gaps


# ---------------------------------------------------------------------------
# Lagrangian seeding into void (Sec. 3.2.1 seeding routine, reading R35)
# ---------------------------------------------------------------------------

def seed_block(dim, n, ramp, bc=0, b=(3e-4, -2e-4, 1e-4), garbage=1.0, Lb=1e-3, p=1e5,
               numax=1.0 - 1e-6):
    """A CuBe block with a void fraction nu = ramp(x, y, z) clipped to
    numax < 1 (the CuBe keeps a trace), at rest at 1e5 Pa, with X = x + b
    where nu <= 1/2
    and X = x + garbage where nu > 1/2; box [0, Lb]^dim, boundary rule bc on
    every side; pressure p."""
    mats = [W.void(), CUBE]
    n3 = [n if k < dim else 1 for k in range(3)]
    hi = [Lb if k < dim else 1.0 for k in range(3)]
    c = W.Case("seed", dim, n3, [0, 0, 0], hi, [bc] * (2 * dim), mats, None, cfl=0.6)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    cen = c.centres()
    nu = np.clip(ramp(*cen[:dim]), 0.0, numax)
    c.prim[lay.o_phi] = nu
    c.prim[lay.o_rho] = 0.0
    c.prim[lay.o_rho + 1] = CUBE["rho0"]
    c.prim[lay.o_p] = p
    for d in range(dim):
        c.prim[lay.o_X + d] = cen[d] + np.where(nu > 0.5, garbage, b[d])
    return c


def _seeded_cells(c, nu):
    """Cells the routine seeds: nu > 1/2 and |grad nu| h > 1e-6 (central
    differences, the boundary rule applied to the neighbours)."""
    lay = c.layout
    dim = c.dim
    A = nu.reshape([c.n[k] for k in range(dim)][::-1])
    g = np.zeros(A.shape)
    for d in range(dim):
        ax = dim - 1 - d
        if c.bc[2 * d] == W.BC_PERIODIC:
            up, dn = np.roll(A, -1, axis=ax), np.roll(A, 1, axis=ax)
        else:
            pad = np.concatenate([np.take(A, [0], axis=ax), A, np.take(A, [-1], axis=ax)], axis=ax)
            up = np.take(pad, range(2, A.shape[ax] + 2), axis=ax)
            dn = np.take(pad, range(0, A.shape[ax]), axis=ax)
        g += ((up - dn) / (2 * c.dx[d])) ** 2
    h = max(c.dx[:dim])
    return ((A > 0.5) & (np.sqrt(g) * h > 1e-6)).reshape(-1)


def _check_seeding(c, rounds, b, lib, tol=1e-12, garbage_deep=True, margin=3):
    if not garbage_deep:
        # garbage only where the routine seeds; the void it leaves alone
        # (nu uniform around it) holds X = x + b
        lay = c.layout
        keep = ~_seeded_cells(c, c.prim[lay.o_phi])
        cen = c.centres()
        for d in range(c.dim):
            c.prim[lay.o_X + d][keep] = cen[d][keep] + b[d]
    g = OracleGrid(c, lib=lib)
    lay = c.layout
    U0 = g.read(False)
    for _ in range(rounds):
        g.seed_x()
    U = g.read(False)
    nu = U0[lay.o_phi]
    seeded = _seeded_cells(c, nu)
    assert seeded.sum() >= 4
    # checked: seeded cells whose probe stencils (and those of the cells
    # they read, round after round) stay off transmissive boundaries: there
    # the ghost copies the edge cell, which does not continue an affine X
    ix = np.indices([c.n[k] for k in range(c.dim)][::-1]).reshape(c.dim, -1)[::-1]
    inner = np.ones(c.ncell, dtype=bool)
    for d in range(c.dim):
        if c.bc[2 * d] == W.BC_TRANSMISSIVE:
            inner &= (ix[d] >= margin) & (ix[d] <= c.n[d] - 1 - margin)
    chk = seeded & inner
    assert chk.sum() >= 4
    cen = c.centres()
    for d in range(c.dim):
        X = U[lay.o_X + d]
        # seeded cells: the material's X continued, c + b, to rounding
        err = np.abs(X[chk] - (cen[d][chk] + b[d])).max()
        assert err <= tol * (c.hi[d] - c.lo[d]), (d, err)
    # every other cell and every other field unchanged bit for bit
    keep = ~seeded
    assert np.array_equal(U[:, keep], U0[:, keep])
    other = [f for f in range(lay.nfield) if not lay.o_X <= f < lay.o_X + c.dim]
    assert np.array_equal(U[other], U0[other])


def _ramp(s, w):
    """nu rising linearly from 0 to 1 over a width w centred at s = 0."""
    return np.clip(0.5 + s / w, 0.0, 1.0)


def check_seeding_continues_affine_x_1d(lib=None):
    """1D: void rising to the right over 8 cells; after six applications
    (each reaches about a cell further from the material) every seeded cell
    holds the material's X = x + b continued (1e-12 of the box)."""
    Lb, n = 1e-3, 64
    c = seed_block(1, n, lambda x: _ramp(x - 0.5 * Lb, 8 * Lb / n), Lb=Lb)
    _check_seeding(c, 6, (3e-4,), lib)


def check_seeding_continues_affine_x_2d(lib=None):
    """2D: the void rises across an oblique line (normal at 30 degrees); the
    probe's bilinear interpolation of X = x + b is exact, so every seeded
    cell holds c + b (1e-12) whatever the numerical normal."""
    Lb, n = 1e-3, 48
    th = np.deg2rad(30.0)
    c = seed_block(2, n, lambda x, y: _ramp(np.cos(th) * (x - 0.5 * Lb) + np.sin(th) * (y - 0.5 * Lb),
                                           8 * Lb / n), Lb=Lb)
    _check_seeding(c, 8, (3e-4, -2e-4), lib)


def check_seeding_continues_affine_x_3d(lib=None):
    """3D: the same across an oblique plane (garbage in the seeded cells
    only: at the top of the ramp the probes' stencils touch void that is
    never seeded; the probe's direction is pinned in 1D and 2D)."""
    Lb, n = 1e-3, 20
    nrm = np.array([0.5, 0.3, 0.81])
    nrm /= np.linalg.norm(nrm)
    c = seed_block(3, n, lambda x, y, z: _ramp(nrm[0] * (x - 0.5 * Lb) + nrm[1] * (y - 0.5 * Lb)
                                               + nrm[2] * (z - 0.5 * Lb), 8 * Lb / n), Lb=Lb)
    _check_seeding(c, 16, (3e-4, -2e-4, 1e-4), lib, garbage_deep=False, margin=6)


def check_seeding_across_periodic_wrap(lib=None):
    """Periodic 1D: the void rises from x = 0 to the right and the material
    lies before the wrap (x near the box's end); probes from the first
    cells cross the wrap, where X continues shifted by the period."""
    Lb, n = 1e-3, 64

    def ramp(x):
        # nu rises through 1/2 at x = 0 (the wrap) and falls back at L/2
        s = np.where(x < 0.5 * Lb, x, x - Lb)
        return _ramp(s, 8 * Lb / n) * _ramp(0.5 * Lb - 4 * Lb / n - x, 8 * Lb / n)
    c = seed_block(1, n, ramp, bc=W.BC_PERIODIC, Lb=Lb)
    _check_seeding(c, 8, (3e-4,), lib)


def check_seeding_across_reflective_wall(lib=None):
    """Reflective 1D: one cell of material at the right wall, the void
    rising away from it to the left, and X = x (b = 0, the only affine X a
    mirror continues): the probes of the cells next to it cross the wall,
    take the mirrored X there, and every seeded cell holds c."""
    Lb, n = 1e-3, 32
    dx = Lb / n
    c = seed_block(1, n, lambda x: _ramp((Lb - 1.2 * dx) - x, 9 * dx), bc=W.BC_REFLECTIVE,
                   b=(0.0,), Lb=Lb)
    _check_seeding(c, 8, (0.0,), lib)


def check_seeding_in_the_step(lib=None):
    """A stress-free block (p = 0 at the reference density, so the void's
    (1 - nu) p puts no force on it) moving at 120 m/s along x into void,
    X = x + b everywhere: seeding before every step keeps the affine X that
    the transport at uniform velocity carries exactly, X = x + b - u t
    after 30 steps (1e-11 of the box)."""
    Lb, n = 1e-3, 64
    c = seed_block(1, n, lambda x: _ramp(x - 0.6 * Lb, 8 * Lb / n), Lb=Lb, garbage=3e-4, p=0.0)
    lay = c.layout
    c.prim[lay.o_u] = 120.0
    g = OracleGrid(c, lib=lib)
    info = g.step(30)
    w = g.read()
    x = c.centres()[0]
    assert _seeded_cells(c, w[lay.o_phi]).sum() >= 4
    # (eight cells from each end: the transmissive ghosts copy the edge,
    # which is not an affine continuation, and that reaches a few cells in)
    err = np.abs(w[lay.o_X][8:-8] - (x[8:-8] + 3e-4 - 120.0 * info["t"])).max()
    assert err <= 1e-11 * Lb, err


CHECKS = {
    "no_opening_in_compression": check_no_opening_in_compression,
    "no_opening_without_critical_damage": check_no_opening_without_critical_damage,
    "release_from_a_crack": check_release_from_a_crack,
    "opening_at_capped_damage": check_opening_at_capped_damage,
    "porous_stress_equilibrium": check_porous_stress_equilibrium,
    "void_opening_mirror": check_void_opening_mirror,
    "void_opening_galilean": check_void_opening_galilean,
    "seeding_continues_affine_x_1d": check_seeding_continues_affine_x_1d,
    "seeding_continues_affine_x_2d": check_seeding_continues_affine_x_2d,
    "seeding_continues_affine_x_3d": check_seeding_continues_affine_x_3d,
    "seeding_across_periodic_wrap": check_seeding_across_periodic_wrap,
    "seeding_across_reflective_wall": check_seeding_across_reflective_wall,
    "seeding_in_the_step": check_seeding_in_the_step,
}


if __name__ == "__main__":
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
