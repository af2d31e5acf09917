"""Small seeded cases used by the oracle pins and by the GPU parity tests
(initial data only; no arithmetic of the method)."""
import numpy as np

from paper_2210_04037_gb300 import workloads as W


def gas_riemann(n, WL, WR, x0=0.5, gamma=1.4):
    mats = [dict(W.air(), gamma_gas=gamma)]
    c = W.Case("riemann", 1, [n, 1, 1], [0, 0, 0], [1, 1, 1], [0, 0], mats, None, cfl=0.6)
    lay = c.layout
    c.prim = W.blank_prim(lay, n)
    x = c.centres()[0]
    left = x < x0
    for k, o in enumerate((lay.o_rho, lay.o_u, lay.o_p)):
        c.prim[o] = np.where(left, WL[k], WR[k])
    c.prim[lay.o_X] = x
    return c


def elastic_cube(n, length, u_of_x, bc=(1, 1), plastic=False, rho_of_x=None):
    """Single-material CuBe bar, F = I, p = 1e5 (damage off)."""
    m = W.cube(damage="none", plastic=plastic)
    c = W.Case("bar", 1, [n, 1, 1], [0, 0, 0], [length, 1, 1], list(bc), [m], None, cfl=0.6)
    lay = c.layout
    c.prim = W.blank_prim(lay, n)
    x = c.centres()[0]
    c.prim[lay.o_rho] = m["rho0"] if rho_of_x is None else rho_of_x(x)
    c.prim[lay.o_u] = u_of_x(x)
    c.prim[lay.o_p] = 1e5
    c.prim[lay.o_X] = x
    return c


def periodic_mix_2d(n, seed=5, shear=0.003, plastic=True, p0=5e8, dp=5e7,
                    rho_gas=700.0, vel=5.0, bc=1):
    """Smooth periodic copper/air mixture under compression (no tension in
    gas-rich cells, where an ideal-gas phase would have unbounded negative
    energy), with a shear that yields; drives the mixture, shear and
    plastic terms."""
    rng = np.random.default_rng(seed)
    mats = [W.cube("bonora", plastic=plastic), W.air()]
    c = W.Case("mix2d", 2, [n, n, 1], [0, 0, 0], [1e-3, 1e-3, 1], [bc] * 4, mats, None, cfl=0.5)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    x, y = c.centres()
    k = 2 * np.pi / 1e-3
    a = rng.uniform(0.5, 1.5, 4)
    frac = 0.5 + 0.45 * np.sin(k * x + a[0]) * np.cos(k * y + a[1])
    W.fill_two_phase(c, frac, 8370.0 * (1 + 0.002 * np.cos(k * y)), rho_gas,
                     p0 + dp * np.sin(k * x + a[2]),
                     [vel * np.sin(k * y + a[3]), vel * np.cos(k * x)])
    c.prim[lay.F_index(0, 1)] = shear * np.sin(k * x)
    return c


def periodic_impact_1d(n, v=150.0):
    """Aluminium flyer onto an aluminium target in air on a periodic line:
    impact, plastic flow and the simple damage law are active."""
    c = spall_like_1d(n, v, solid=W.al_h32("simple"))
    c.bc = [1, 1]
    return c


def spall_like_1d(n, v=150.0, solid=None):
    """Copper flyer onto a copper target in air (plastic + Bonora damage),
    transmissive ends; a small 1D impact used for symmetry tests."""
    mats = [W.cube("bonora") if solid is None else solid, W.air()]
    c = W.Case("imp1d", 1, [n, 1, 1], [0, 0, 0], [2e-3, 1, 1], [0, 0], mats, None, cfl=0.6)
    lay = c.layout
    c.prim = W.blank_prim(lay, n)
    x = c.centres()[0]
    frac = np.where((x > 0.2e-3) & (x < 1.8e-3), 1.0, 0.0)
    W.fill_two_phase(c, frac, mats[0]["rho0"], 1.2, 1e5, [np.where(x < 0.8e-3, v, 0.0)])
    return c


def _mirror_fields(case, U):
    """Mirror a [nfield, ncell] array of conserved or primitive fields about
    the x mid-plane of the box."""
    lay = case.layout
    n = list(case.n)[: case.dim]
    A = U.reshape([lay.nfield] + n[::-1])[..., ::-1].reshape(lay.nfield, -1).copy()
    A[lay.o_u] *= -1.0
    for c_ in W.F_COMPS[case.dim]:
        i, j = divmod(c_, 3)
        if (i == 0) != (j == 0):
            A[lay.F_index(i, j)] *= -1.0
    A[lay.o_X] = (case.lo[0] + case.hi[0]) - A[lay.o_X]
    return A


def mirrored_x(case):
    import copy
    m = copy.deepcopy(case)
    m.prim = _mirror_fields(case, case.prim)
    m.bc = [case.bc[1], case.bc[0]] + list(case.bc[2:])
    assert case.phi0 is None
    return m


def mirror_back_x(case, U):
    return _mirror_fields(case, U)


def periodic_mix_3d(n, seed=6, shear=0.03, p0=5e8, dp=5e7, rho_gas=700.0, vel=5.0, bc=1,
                    nz=None):
    """3D version of the compressed periodic copper/air mixture: every
    transport term, both tangential directions of the Riemann solver and
    the plastic return are active; no dilute tensile phase."""
    rng = np.random.default_rng(seed)
    nz = n if nz is None else nz
    mats = [W.cube("bonora"), W.air()]
    L = 1e-3
    c = W.Case("mix3d", 3, [n, n + 2, nz], [0, 0, 0], [L, L * (n + 2) / n, L * nz / n], [bc] * 6,
               mats, None, cfl=0.5)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    x, y, z = c.centres()
    k = 2 * np.pi / L
    a = rng.uniform(0.5, 1.5, 6)
    frac = 0.5 + 0.45 * np.sin(k * x + a[0]) * np.cos(k * y + a[1]) * np.cos(k * z * n / nz + a[4])
    W.fill_two_phase(c, frac, 8370.0 * (1 + 0.002 * np.cos(k * y)), rho_gas,
                     p0 + dp * np.sin(k * x + a[2]),
                     [vel * np.sin(k * y + a[3]), vel * np.cos(k * x), vel * np.sin(k * x + a[5])])
    c.prim[lay.F_index(0, 1)] = shear * np.sin(k * x)
    c.prim[lay.F_index(2, 0)] = 0.5 * shear * np.cos(k * y)
    return c
