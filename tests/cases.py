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
                    rho_gas=700.0, vel=5.0, bc=1, solid=None):
    """Smooth periodic copper (or `solid`)/air mixture under compression (no
    tension in gas-rich cells, where an ideal-gas phase would have unbounded
    negative energy), with a shear that yields; drives the mixture, shear
    and plastic terms."""
    rng = np.random.default_rng(seed)
    mats = [W.cube("bonora", plastic=plastic) if solid is None else solid, W.air()]
    c = W.Case("mix2d", 2, [n, n, 1], [0, 0, 0], [1e-3, 1e-3, 1], [bc] * 4, mats, None, cfl=0.5)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    x, y = c.centres()
    k = 2 * np.pi / 1e-3
    a = rng.uniform(0.5, 1.5, 4)
    frac = 0.5 + 0.45 * np.sin(k * x + a[0]) * np.cos(k * y + a[1])
    W.fill_two_phase(c, frac, mats[0]["rho0"] * (1 + 0.002 * np.cos(k * y)), rho_gas,
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


def shear_bar_2d(n, length, uy_of_x, left=None, right=None, x0=None, bc=(0, 0), ux=0.0):
    """A bar along x on an n x 2 grid, periodic in y, moving at ux along x
    (default at rest) with a transverse velocity u_y(x) and Fbar = I,
    p = 1e5 Pa, elastic (no
    plasticity, no damage).  One material (CuBe) by default; with `right`
    given, two materials: `left` for x < x0 and `right` beyond, each at its
    reference density (a bimaterial interface, volume fractions 1 - 1e-6 /
    1e-6)."""
    left = W.cube(damage="none", plastic=False) if left is None else left
    mats = [left] if right is None else [left, right]
    dy = length / n
    c = W.Case("shear", 2, [n, 2, 1], [0, 0, 0], [length, 2 * dy, 1], list(bc) + [1, 1], mats,
               None, cfl=0.6)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    x, y = c.centres()
    if right is None:
        c.prim[lay.o_rho] = left["rho0"]
    else:
        W.fill_two_phase(c, np.where(x < x0, 1.0, 0.0), left["rho0"], right["rho0"], 1e5,
                         [0 * x, 0 * x])
    c.prim[lay.o_u] = ux
    c.prim[lay.o_u + 1] = uy_of_x(x)
    c.prim[lay.o_p] = 1e5
    c.prim[lay.o_X] = x
    c.prim[lay.o_X + 1] = y
    return c


def mirror_fields(case, U, axis, wall2):
    """Mirror a [nfield, ncell] array of conserved or primitive fields along
    `axis`: cells reversed, u_axis and the Fbar comps with exactly one index
    equal to `axis` negated, X_axis -> wall2 - X_axis (wall2: twice the
    mirror plane's coordinate)."""
    lay = case.layout
    n = list(case.n)[: case.dim]
    A = U.reshape([lay.nfield] + n[::-1])
    A = np.flip(A, axis=case.dim - axis).reshape(lay.nfield, -1).copy()
    A[lay.o_u + axis] *= -1.0
    for c_ in W.F_COMPS[case.dim]:
        i, j = divmod(c_, 3)
        if (i == axis) != (j == axis):
            A[lay.F_index(i, j)] *= -1.0
    A[lay.o_X + axis] = wall2 - A[lay.o_X + axis]
    return A


def mirrored(case, axis):
    """The case mirrored about the mid-plane of its box along `axis` (the
    boundary conditions of the two ends swapped)."""
    import copy
    assert case.phi0 is None
    m = copy.deepcopy(case)
    m.prim = mirror_fields(case, case.prim, axis, case.lo[axis] + case.hi[axis])
    bc = list(case.bc)
    bc[2 * axis], bc[2 * axis + 1] = bc[2 * axis + 1], bc[2 * axis]
    m.bc = bc
    return m


def doubled_periodic(case, axis):
    """The box [lo, hi] along `axis` doubled to [lo, 2 hi - lo] by its mirror
    image about hi, periodic along `axis` (its other boundaries kept): by
    symmetry its half [lo, hi] evolves as the original box with reflective
    walls at both ends."""
    import copy
    assert case.phi0 is None
    d = copy.deepcopy(case)
    lay = case.layout
    n = list(case.n)[: case.dim]
    A = case.prim.reshape([lay.nfield] + n[::-1])
    B = mirror_fields(case, case.prim, axis, 2.0 * case.hi[axis]).reshape(A.shape)
    d.prim = np.concatenate([A, B], axis=case.dim - axis).reshape(lay.nfield, -1).copy()
    nn = list(case.n)
    nn[axis] *= 2
    d.n = nn
    hi = list(case.hi)
    hi[axis] = 2 * case.hi[axis] - case.lo[axis]
    d.hi = hi
    bc = list(case.bc)
    bc[2 * axis] = bc[2 * axis + 1] = W.BC_PERIODIC
    d.bc = bc
    return d


def first_half(case, U, axis):
    """Cells of the first half along `axis` of a doubled box's fields."""
    lay = case.layout
    n = list(case.n)[: case.dim]
    A = U.reshape([lay.nfield] + n[::-1])
    sl = [slice(None)] * (case.dim + 1)
    sl[case.dim - axis] = slice(0, n[axis] // 2)
    return A[tuple(sl)].reshape(lay.nfield, -1)


def embed_3d(case, perm, thin=2):
    """A 1D or 2D case laid into a 3D grid: its axis k becomes axis perm[k]
    of the 3D grid; the remaining axes are `thin` cells wide, periodic and
    uniform.  Velocities, the deformation tensor (Fbar_ij ->
    Fbar_perm(i)perm(j)) and X follow the permutation; the transverse X are
    the cell centres."""
    lay = case.layout
    full = list(perm) + [a for a in range(3) if a not in perm]
    n3, lo3, hi3, bc3 = [thin] * 3, [0.0] * 3, [0.0] * 3, [W.BC_PERIODIC] * 6
    dxs = case.dx
    for k in range(3):
        a = full[k]
        if k < case.dim:
            n3[a], lo3[a], hi3[a] = case.n[k], case.lo[k], case.hi[k]
            bc3[2 * a], bc3[2 * a + 1] = case.bc[2 * k], case.bc[2 * k + 1]
        else:
            lo3[a], hi3[a] = 0.0, thin * dxs[0]
    c3 = W.Case(case.name + "_3d", 3, n3, lo3, hi3, bc3, case.materials, None, cfl=case.cfl)
    l3 = c3.layout
    w3 = W.blank_prim(l3, c3.ncell)
    # source cell of each 3D cell: its coordinates along the case's axes
    idx3 = np.meshgrid(*[np.arange(n3[a]) for a in range(3)][::-1], indexing="ij")[::-1]
    idx3 = [g.reshape(-1) for g in idx3]
    src = np.zeros(c3.ncell, dtype=np.int64)
    stride = 1
    for k in range(case.dim):
        src += idx3[full[k]] * stride
        stride *= case.n[k]
    P = case.prim[:, src]
    for f in range(lay.o_u):
        w3[f] = P[f]
    w3[l3.o_p] = P[lay.o_p]
    for k in range(case.dim):
        w3[l3.o_u + full[k]] = P[lay.o_u + k]
        w3[l3.o_X + full[k]] = P[lay.o_X + k]
    cen = c3.centres()
    for k in range(case.dim, 3):
        w3[l3.o_X + full[k]] = cen[full[k]]
    for c_ in W.F_COMPS[case.dim]:
        i, j = divmod(c_, 3)
        w3[l3.F_index(full[i], full[j])] = P[lay.F_index(i, j)]
    for h in range(2 * lay.nhist):
        w3[l3.o_hist + h] = P[lay.o_hist + h]
    c3.prim = w3
    return c3, full, src


def unembed_3d(case, c3, full, U3, src):
    """Fields of a 3D run of `embed_3d(case, ...)` mapped back to the case's
    layout, one 3D cell per case cell (the first of its transverse copies)."""
    lay, l3 = case.layout, c3.layout
    first = np.full(case.ncell, -1, dtype=np.int64)
    for c in range(c3.ncell - 1, -1, -1):
        first[src[c]] = c
    Q = U3[:, first]
    out = np.zeros((lay.nfield, case.ncell))
    for f in range(lay.o_u):
        out[f] = Q[f]
    out[lay.o_p] = Q[l3.o_p]
    for k in range(case.dim):
        out[lay.o_u + k] = Q[l3.o_u + full[k]]
        out[lay.o_X + k] = Q[l3.o_X + full[k]]
    for c_ in W.F_COMPS[case.dim]:
        i, j = divmod(c_, 3)
        out[lay.F_index(i, j)] = Q[l3.F_index(full[i], full[j])]
    for h in range(2 * lay.nhist):
        out[lay.o_hist + h] = Q[l3.o_hist + h]
    return out


def cracked_block(dim, n, p=-2e8, vel=5.0, seed=0, with_void=True, bc=0):
    """A CuBe block in hydrostatic tension p (negative) with one plane of
    critically damaged cells (D = D_crit) across the middle of each axis (a
    cross in 2D, three planes in 3D), so that void opens across faces of
    every axis; a smooth seeded velocity perturbation of amplitude `vel`;
    with `with_void` a void material (fraction 0, density 0) as material 0
    before the CuBe.  Transmissive (bc=0) or periodic (bc=1) on every side."""
    rng = np.random.default_rng(seed)
    cube = W.cube("bonora")
    mats = [W.void(), cube] if with_void else [cube]
    L = 1e-3
    n3 = [n if k < dim else 1 for k in range(3)]
    hi = [L if k < dim else 1.0 for k in range(3)]
    c = W.Case("cracked", dim, n3, [0, 0, 0], hi, [bc] * (2 * dim), mats, None, cfl=0.6)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    cen = c.centres()
    k = 1 if with_void else 0
    if with_void:
        c.prim[lay.o_phi] = 0.0
        c.prim[lay.o_rho] = 0.0
    c.prim[lay.o_rho + k] = cube["rho0"]
    kk = 2 * np.pi / L
    a = rng.uniform(0.0, 2 * np.pi, 2 * dim)
    for d in range(dim):
        other = cen[(d + 1) % dim]
        c.prim[lay.o_u + d] = vel * np.sin(kk * cen[d] + a[d]) * np.cos(kk * other + a[dim + d])
    c.prim[lay.o_p] = p
    crack = np.zeros(c.ncell, dtype=bool)
    dx = L / n
    for d in range(dim):
        crack |= np.abs(cen[d] - (0.5 * L + 0.5 * dx)) < 0.5 * dx
    c.prim[lay.o_hist + 1] = np.where(crack, cube["D_crit"], 0.0)
    for d in range(dim):
        c.prim[lay.o_X + d] = cen[d]
    return c


def three_mix_2d(n, seed=8, shear=0.02, p0=5e8, dp=5e7, vel=5.0, bc=1):
    """Smooth periodic mixture of two plastic solids and a gas (Al-H32,
    CuBe with Bonora damage, air at 700 kg/m^3) under compression, with a
    shear that yields: the two-plastic closure in 2D."""
    rng = np.random.default_rng(seed)
    mats = [W.al_h32("none"), W.cube("bonora"), W.air()]
    c = W.Case("mix3m", 2, [n, n, 1], [0, 0, 0], [1e-3, 1e-3, 1], [bc] * 4, mats, None, cfl=0.5)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    x, y = c.centres()
    k = 2 * np.pi / 1e-3
    a = rng.uniform(0.5, 1.5, 5)
    f_al = 0.3 + 0.2 * np.sin(k * x + a[0]) * np.cos(k * y + a[1])
    f_cu = 0.3 + 0.2 * np.cos(k * x + a[2]) * np.sin(k * y)
    c.prim[lay.o_phi] = f_al
    c.prim[lay.o_phi + 1] = f_cu
    c.prim[lay.o_rho] = mats[0]["rho0"] * (1 + 0.002 * np.cos(k * y))
    c.prim[lay.o_rho + 1] = mats[1]["rho0"] * (1 + 0.002 * np.sin(k * x))
    c.prim[lay.o_rho + 2] = 700.0
    c.prim[lay.o_u] = vel * np.sin(k * y + a[3])
    c.prim[lay.o_u + 1] = vel * np.cos(k * x)
    c.prim[lay.o_p] = p0 + dp * np.sin(k * x + a[4])
    c.prim[lay.F_index(0, 1)] = shear * np.sin(k * x)
    c.prim[lay.o_X] = x
    c.prim[lay.o_X + 1] = y
    return c
