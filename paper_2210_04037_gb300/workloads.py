"""Seeded synthetic inputs: material tables, the perturbation lattice and the
initial primitive fields of each workload.

This module holds no arithmetic of the method itself (no equation of state,
no flux, no source): it only lays out initial data.  It serves both the CUDA
path and the CPU oracle, which each convert the primitive fields to their own
conserved state.

Field order (shared by the initial data, ``mm_read_fields`` and the oracle),
for ``dim`` space dimensions, ``N`` materials and ``H`` plastic materials:

    phi_0 .. phi_{N-2}            volume fractions (phi_{N-1} = 1 - sum)
    rho_0 .. rho_{N-1}            phasic densities      (conserved: phi_l rho_l)
    u_0 .. u_{dim-1}              velocity              (conserved: rho u)
    p                             mixture pressure      (conserved: rho E)
    Fbar comps                    unimodular deformation tensor, row-major:
                                  dim 1: xx yy zz; dim 2: xx xy yx yy zz;
                                  dim 3: all nine
    (eps_p, D) per plastic mat.   plastic strain, damage (conserved: x phi rho)
    X_0 .. X_{dim-1}              Lagrangian coordinates

Material parameters are those of the paper's tables (Romenskii EOS table,
Johnson-Cook table, Bonora table; Sec. 4.3 for the simple damage model).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np

BC_TRANSMISSIVE, BC_PERIODIC, BC_REFLECTIVE = 0, 1, 2
FP64, FP32_SPLIT = 0, 1
PHI_MIN = 1e-6

# --------------------------------------------------------------------------
# material tables
# --------------------------------------------------------------------------

MATERIAL_KEYS = ("eos", "rho0", "K0", "G0", "alpha", "beta", "Gamma0",
                 "gamma_gas", "plasticity", "c1", "c2", "c3", "n_hard",
                 "edot0", "damage", "D_crit", "eps_t", "eps_c", "alpha_D",
                 "poisson", "Ddot0", "shear_model", "Gp", "Gamma1", "Gamma2",
                 "gamma_s")
SHEAR_ROMENSKII, SHEAR_STEINBERG = 0, 1


def material(**kw) -> Dict[str, float]:
    m = {k: 0.0 for k in MATERIAL_KEYS}
    m.update(eos=0, plasticity=0, damage=0, edot0=1.0, gamma_gas=1.4, shear_model=0)
    m.update(kw)
    return m


def air() -> Dict[str, float]:
    """Ideal-gas air (gamma 1.4); the paper gives no gas parameters."""
    return material(eos=0, rho0=1.2, gamma_gas=1.4)


def cube(damage: str = "bonora", plastic: bool = True) -> Dict[str, float]:
    """CuBe: Romenskii row, Johnson-Cook row (no thermal term), Bonora row."""
    m = material(eos=1, rho0=8370.0, K0=131.3e9, G0=53.6e9, alpha=1.0,
                 beta=3.0, Gamma0=2.0)
    if plastic:
        m.update(plasticity=1, c1=1.041e9, c2=0.0, c3=0.025, n_hard=0.31)
    if damage == "bonora" and plastic:
        m.update(damage=1, D_crit=0.85, eps_t=0.08, eps_c=0.16, alpha_D=0.631,
                 poisson=0.324)
    return m


def al_h32(damage: str = "simple", plastic: bool = True) -> Dict[str, float]:
    """Al-H32: Romenskii row, Johnson-Cook row; the simple damage model of the
    expanding-ring test (Ddot0 = 0.15, D_crit = 0.1), since Al has no Bonora
    row."""
    m = material(eos=1, rho0=2670.0, K0=72.2e9, G0=25.8e9, alpha=0.627354,
                 beta=2.28816, Gamma0=1.48389)
    if plastic:
        m.update(plasticity=1, c1=0.275e9, c2=0.114e9, c3=0.002, n_hard=0.42)
    if damage == "simple" and plastic:
        m.update(damage=2, Ddot0=0.15, D_crit=0.1)
    return m


def u_nb(damage: str = "simple", plastic: bool = True) -> Dict[str, float]:
    """U-Nb: the Romenskii cold energy with the Steinberg shear modulus
    G = G0 + Gp p_c eta^(-1/3) and Gamma = Gamma0 + Gamma1 eta^(-1/3) +
    Gamma2 eta^(-gamma) (Romenskii-Steinberg row), Johnson-Cook row (no
    thermal term), the simple damage model of the expanding-ring test
    (Ddot0 = 0.15, D_crit = 0.1, Sec. 4.3)."""
    m = material(eos=1, rho0=17411.0, K0=111.27e9, G0=26.34e9, alpha=1.105,
                 Gamma0=0.5, shear_model=SHEAR_STEINBERG, Gp=1.1226, Gamma1=1.056,
                 Gamma2=1.068, gamma_s=3.843)
    if plastic:
        m.update(plasticity=1, c1=0.780e9, c2=0.253e9, c3=0.012, n_hard=0.22)
    if damage == "simple" and plastic:
        m.update(damage=2, Ddot0=0.15, D_crit=0.1)
    return m


def void() -> Dict[str, float]:
    """The void volume fraction nu of Sec. 2.1, carried as a material of its
    own (eos 2): no mass, no energy, no stress; it takes the volume a
    void-opening face creates (Sec. 3.1).  Never the last material."""
    return material(eos=2, rho0=0.0)


def steel_304l_disk() -> Dict[str, float]:
    """304L: Romenskii row, Johnson-Cook hardening/rate (thermal term not
    modelled), Bonora row of the expanding-disk test."""
    return material(eos=1, rho0=8000.0, K0=158.3e9, G0=73.1e9, alpha=0.569,
                    beta=2.437, Gamma0=1.84, plasticity=1, c1=0.253e9,
                    c2=0.685e9, c3=0.097, n_hard=0.313, damage=1, D_crit=0.3,
                    eps_t=0.002, eps_c=0.5, alpha_D=0.5, poisson=0.3)


# --------------------------------------------------------------------------
# layout
# --------------------------------------------------------------------------

F_COMPS = {1: (0, 4, 8), 2: (0, 1, 3, 4, 8), 3: tuple(range(9))}


@dataclasses.dataclass(frozen=True)
class Layout:
    dim: int
    nmat: int
    nhist: int

    @property
    def nF(self) -> int:
        return len(F_COMPS[self.dim])

    @property
    def o_phi(self) -> int:
        return 0

    @property
    def o_rho(self) -> int:
        return self.nmat - 1

    @property
    def o_u(self) -> int:
        return self.o_rho + self.nmat

    @property
    def o_p(self) -> int:
        return self.o_u + self.dim

    @property
    def o_F(self) -> int:
        return self.o_p + 1

    @property
    def o_hist(self) -> int:
        return self.o_F + self.nF

    @property
    def o_X(self) -> int:
        return self.o_hist + 2 * self.nhist

    @property
    def nfield(self) -> int:
        return self.o_X + self.dim

    def F_index(self, i: int, j: int) -> Optional[int]:
        c = 3 * i + j
        comps = F_COMPS[self.dim]
        return self.o_F + comps.index(c) if c in comps else None

    def names(self) -> List[str]:
        out = [f"phi{l}" for l in range(self.nmat - 1)]
        out += [f"rho{l}" for l in range(self.nmat)]
        out += [f"u{k}" for k in range(self.dim)]
        out += ["p"]
        out += [f"F{c // 3}{c % 3}" for c in F_COMPS[self.dim]]
        for h in range(self.nhist):
            out += [f"eps{h}", f"D{h}"]
        out += [f"X{k}" for k in range(self.dim)]
        return out

    def cons_names(self) -> List[str]:
        out = [f"phi{l}" for l in range(self.nmat - 1)]
        out += [f"arho{l}" for l in range(self.nmat)]
        out += [f"mom{k}" for k in range(self.dim)]
        out += ["rhoE"]
        out += [f"F{c // 3}{c % 3}" for c in F_COMPS[self.dim]]
        for h in range(self.nhist):
            out += [f"areps{h}", f"arhoD{h}"]
        out += [f"X{k}" for k in range(self.dim)]
        return out


# --------------------------------------------------------------------------
# counter-based random numbers: splitmix64 (Steele, Lea & Flood 2014)
# --------------------------------------------------------------------------

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream of ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def gaussian(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    u = uniform01(seed, 2 * count)
    u1, u2 = 1.0 - u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def perturbation_uniform(seed: int, shape: Sequence[int], a: float) -> np.ndarray:
    """phi0 ~ U(1-a, 1+a) (Sec. 3.2.2)."""
    n = int(np.prod(shape))
    return (1.0 - a + 2.0 * a * uniform01(seed, n)).astype(np.float32)


def perturbation_gaussian(seed: int, shape: Sequence[int], sd: float) -> np.ndarray:
    """phi0 ~ rectified N(1, sd^2): negative draws set to 0 (Sec. 3.2.2)."""
    n = int(np.prod(shape))
    return np.maximum(1.0 + sd * gaussian(seed, n), 0.0).astype(np.float32)


# --------------------------------------------------------------------------
# case description
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Case:
    name: str
    dim: int
    n: Sequence[int]
    lo: Sequence[float]
    hi: Sequence[float]
    bc: Sequence[int]              # [dim*2]: (lo, hi) per axis
    materials: List[Dict[str, float]]
    prim: np.ndarray               # [nfield, ncell] float64
    phi0: Optional[np.ndarray] = None   # float32, x fastest
    pn: Sequence[int] = (0, 0, 0)
    plo: Sequence[float] = (0.0, 0.0, 0.0)
    ph: Sequence[float] = (1.0, 1.0, 1.0)
    cfl: float = 0.6
    steps: int = 100

    @property
    def layout(self) -> Layout:
        nh = sum(1 for m in self.materials if m["plasticity"] == 1)
        return Layout(self.dim, len(self.materials), nh)

    @property
    def ncell(self) -> int:
        return int(np.prod(list(self.n)[: self.dim]))

    @property
    def dx(self) -> List[float]:
        return [(self.hi[k] - self.lo[k]) / self.n[k] for k in range(self.dim)]

    def centres(self) -> List[np.ndarray]:
        """Cell-centre coordinates, each flattened with x fastest."""
        axes = [self.lo[k] + (np.arange(self.n[k]) + 0.5) * self.dx[k]
                for k in range(self.dim)]
        grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
        return [g.reshape(-1) for g in grids]


def blank_prim(lay: Layout, ncell: int) -> np.ndarray:
    w = np.zeros((lay.nfield, ncell))
    for k in range(3):
        idx = lay.F_index(k, k)
        if idx is not None:
            w[idx] = 1.0
    return w


def fill_two_phase(case: Case, frac_solid: np.ndarray, rho_solid: float,
                   rho_gas: float, p: float, vel: Sequence[np.ndarray]) -> None:
    """Solid is material 0, gas material 1; X set to the cell centres."""
    lay = case.layout
    w = case.prim
    w[lay.o_phi] = np.clip(frac_solid, PHI_MIN, 1.0 - PHI_MIN)
    w[lay.o_rho] = rho_solid
    w[lay.o_rho + 1] = rho_gas
    for k in range(case.dim):
        w[lay.o_u + k] = vel[k]
    w[lay.o_p] = p
    for k, c in enumerate(case.centres()):
        w[lay.o_X + k] = c


def _coverage_1d(lo_cell: np.ndarray, hi_cell: np.ndarray, a: float, b: float) -> np.ndarray:
    ov = np.minimum(hi_cell, b) - np.maximum(lo_cell, a)
    return np.clip(ov / (hi_cell - lo_cell), 0.0, 1.0)


def _annulus_fraction(x: np.ndarray, y: np.ndarray, dx: float, r0: float,
                      r1: float, sub: int) -> np.ndarray:
    f = np.zeros_like(x)
    offs = (np.arange(sub) + 0.5) / sub - 0.5
    for ox in offs:
        for oy in offs:
            r = np.hypot(x + ox * dx, y + oy * dx)
            f += ((r >= r0) & (r <= r1)).astype(np.float64)
    return f / (sub * sub)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def spall_1d(ncell: int = 1000, seed: int = 1, sd: float = 0.05,
             v_flyer: float = 300.0) -> Case:
    """1D plate impact: copper flyer 2 mm at 300 m/s onto a 6 mm copper
    target at rest, gas either side, on [0, 11] mm (the spall domain of
    Sec. 4.1); transmissive ends; phi0 rectified N(1, sd^2) per cell."""
    mats = [cube("bonora"), air()]
    case = Case("spall_1d", 1, [ncell, 1, 1], [0.0, 0, 0], [0.011, 1, 1],
                [BC_TRANSMISSIVE] * 2, mats, None, cfl=0.6, steps=2000)
    case.prim = blank_prim(case.layout, ncell)
    dx = case.dx[0]
    edges = np.arange(ncell + 1) * dx
    frac = _coverage_1d(edges[:-1], edges[1:], 0.001, 0.009)
    x = case.centres()[0]
    u = np.where((x >= 0.001) & (x < 0.003), v_flyer, 0.0)
    fill_two_phase(case, frac, 8370.0, 1.2, 1.0e5, [u])
    case.phi0 = perturbation_gaussian(seed, [ncell], sd)
    case.pn, case.plo, case.ph = [ncell, 1, 1], [0.5 * dx, 0, 0], [dx, 1, 1]
    return case


def spall_al_cube_1d(ncell: int = 1000, seed: int = 1, a: float = 0.0,
                     v_flyer: float = 300.0) -> Case:
    """The 1D spallation test of Sec. 4.1 with its three materials: an
    Al-H32 flyer (Al 5083 H32: Romenskii and Johnson-Cook rows, no damage)
    2 mm thick at v_flyer onto a 6 mm CuBe target at rest (Bonora damage),
    air either side at 1e5 Pa, on [0, 11] mm; transmissive ends; the CuBe's
    yield stress perturbed by phi0 ~ U(1 - a, 1 + a) per cell (a = 0: none).
    Volume fractions from exact cell coverage, clipped to [1e-6, 1 - 1e-6]
    with the air taking the rest."""
    al, cu, gas = al_h32("none"), cube("bonora"), air()
    mats = [al, cu, gas]
    case = Case("spall_al_cube_1d", 1, [ncell, 1, 1], [0.0, 0, 0], [0.011, 1, 1],
                [BC_TRANSMISSIVE] * 2, mats, None, cfl=0.6, steps=2000)
    lay = case.layout
    case.prim = blank_prim(lay, ncell)
    dx = case.dx[0]
    edges = np.arange(ncell + 1) * dx
    f_al = _coverage_1d(edges[:-1], edges[1:], 0.001, 0.003)
    f_cu = _coverage_1d(edges[:-1], edges[1:], 0.003, 0.009)
    f_al = np.clip(f_al, PHI_MIN, 1.0 - 2 * PHI_MIN)
    f_cu = np.clip(f_cu, PHI_MIN, 1.0 - f_al - PHI_MIN)
    case.prim[lay.o_phi] = f_al
    case.prim[lay.o_phi + 1] = f_cu
    case.prim[lay.o_rho] = al["rho0"]
    case.prim[lay.o_rho + 1] = cu["rho0"]
    case.prim[lay.o_rho + 2] = gas["rho0"]
    x = case.centres()[0]
    case.prim[lay.o_u] = np.where(f_al > 0.5, v_flyer, 0.0)
    case.prim[lay.o_p] = 1.0e5
    case.prim[lay.o_X] = x
    if a > 0:
        case.phi0 = perturbation_uniform(seed, [ncell], a)
        case.pn, case.plo, case.ph = [ncell, 1, 1], [0.5 * dx, 0, 0], [dx, 1, 1]
    return case


def ring_2d(n: int = 512, seed: int = 2, a: float = 0.1, v: float = 200.0,
            width: float = 0.064, r0: float = 0.020, r1: float = 0.024,
            lattice_h: float = 0.0005, solid: Optional[Dict[str, float]] = None,
            sd: Optional[float] = None) -> Case:
    """2D expanding ring: Al-H32 (or `solid`) annulus r0..r1 with radial
    velocity v in ideal-gas air at rest, 1e5 Pa; simple damage; phi0 ~
    U(1-a, 1+a) (or, with sd given, rectified N(1, sd^2)) on a lattice of
    spacing lattice_h covering the annulus."""
    mats = [al_h32("simple") if solid is None else solid, air()]
    half = 0.5 * width
    case = Case("ring_2d", 2, [n, n, 1], [-half, -half, 0], [half, half, 1],
                [BC_TRANSMISSIVE] * 4, mats, None, cfl=0.6, steps=100)
    case.prim = blank_prim(case.layout, case.ncell)
    x, y = case.centres()
    frac = _annulus_fraction(x, y, case.dx[0], r0, r1, 4)
    r = np.hypot(x, y)
    inside = frac >= 0.5
    rs = np.where(r > 0, r, 1.0)
    fill_two_phase(case, frac, mats[0]["rho0"], 1.2, 1.0e5,
                   [np.where(inside, v * x / rs, 0.0), np.where(inside, v * y / rs, 0.0)])
    ext = r1 + 2 * lattice_h
    m = int(np.ceil(2 * ext / lattice_h)) + 1
    case.phi0 = (perturbation_uniform(seed, [m, m], a) if sd is None
                 else perturbation_gaussian(seed, [m, m], sd))
    case.pn, case.plo, case.ph = [m, m, 1], [-ext, -ext, 0], [lattice_h, lattice_h, 1]
    return case


def ring_unb_2d(n: int = 256, seed: int = 21, v: float = 210.0) -> Case:
    """The expanding U-Nb ring of Sec. 4.3 in 2D: the annulus 17.185 ..
    17.945 mm of U-Nb (Steinberg closure, simple damage) in air on the
    +-30 mm box, moving radially at v (the driver's first speed; the rigid
    driver itself is not modelled), phi0 rectified N(1, 0.167^2)."""
    c = ring_2d(n, seed=seed, v=v, width=0.060, r0=0.017185, r1=0.017945, solid=u_nb("simple"),
                sd=0.167)
    c.name = "ring_unb_2d"
    return c


def cylinder_3d(n: int = 256, seed: int = 3, sd: float = 0.1, v: float = 250.0,
                width: float = 0.0512, r0: float = 0.018, r1: float = 0.020,
                lattice_h: float = 0.0005, nz: Optional[int] = None) -> Case:
    """3D expanding thin cylinder: CuBe shell r0..r1 about z with radial
    velocity v in ideal-gas air; periodic in z, transmissive in x and y;
    phi0 rectified N(1, sd^2) on a lattice of spacing lattice_h."""
    mats = [cube("bonora"), air()]
    half = 0.5 * width
    nz = n if nz is None else nz
    hz = half * nz / n
    case = Case("cylinder_3d", 3, [n, n, nz], [-half, -half, -hz], [half, half, hz],
                [BC_TRANSMISSIVE] * 4 + [BC_PERIODIC] * 2, mats, None, cfl=0.6,
                steps=500)
    case.prim = blank_prim(case.layout, case.ncell)
    x, y, z = case.centres()
    frac = _annulus_fraction(x, y, case.dx[0], r0, r1, 2)
    r = np.hypot(x, y)
    inside = frac >= 0.5
    rs = np.where(r > 0, r, 1.0)
    fill_two_phase(case, frac, mats[0]["rho0"], 1.2, 1.0e5,
                   [np.where(inside, v * x / rs, 0.0), np.where(inside, v * y / rs, 0.0),
                    np.zeros_like(z)])
    ext = r1 + 2 * lattice_h
    m = int(np.ceil(2 * ext / lattice_h)) + 1
    mz = int(np.ceil(2 * (hz + lattice_h) / lattice_h)) + 1
    case.phi0 = perturbation_gaussian(seed, [m, m, mz], sd)
    case.pn = [m, m, mz]
    case.plo = [-ext, -ext, -(hz + lattice_h)]
    case.ph = [lattice_h] * 3
    return case


def _stratified(seed: int, k: int, jitter: float = 0.6) -> np.ndarray:
    """k positions in [0, 1): one per stratum, jittered by +-jitter/2 of it."""
    return np.mod((np.arange(k) + jitter * (uniform01(seed, k) - 0.5)) / k, 1.0)


def _crack_mask(case: Case, r: np.ndarray, theta: np.ndarray, angles: np.ndarray,
                zc: np.ndarray, z: Optional[np.ndarray], half: float) -> np.ndarray:
    """Cells whose centre lies within `half` of a radial crack plane (angles)
    or of a crack plane z = const (zc, periodic in z)."""
    m = np.zeros(theta.shape, dtype=bool)
    for a in angles:
        d = np.abs(np.mod(theta - a + np.pi, 2.0 * np.pi) - np.pi)
        m |= (d * r < half) & (d < 0.5 * np.pi)
    if z is not None and len(zc):
        L = case.hi[2] - case.lo[2]
        for c in zc:
            d = np.abs(np.mod(z - c + 0.5 * L, L) - 0.5 * L)
            m |= d < half
    return m


def add_void(case: Case, index: int = 1) -> Case:
    """The same case with a void material (no void yet: fraction 0, density
    0) inserted as material `index` (not the last): a grid that can open
    void where critically damaged faces are in tension (Sec. 3.1)."""
    import copy
    nmat = len(case.materials)
    assert 0 <= index < nmat
    out = copy.deepcopy(case)
    out.materials = case.materials[:index] + [void()] + case.materials[index:]
    lay0, lay1 = case.layout, out.layout
    w0 = case.prim
    w1 = np.zeros((lay1.nfield, case.ncell))
    phis = [w0[lay0.o_phi + l] for l in range(nmat - 1)]
    rhos = [w0[lay0.o_rho + l] for l in range(nmat)]
    zero = np.zeros(case.ncell)
    phis = phis[:index] + [zero] + phis[index:]
    rhos = rhos[:index] + [zero] + rhos[index:]
    for l, v in enumerate(phis):
        w1[lay1.o_phi + l] = v
    for l, v in enumerate(rhos):
        w1[lay1.o_rho + l] = v
    w1[lay1.o_u:] = w0[lay0.o_u:]
    out.prim = w1
    out.name = case.name + "_void"
    return out


def expanding_plate(n: int = 512, dim: int = 2, rate: float = 2e5, L: float = 1e-3,
                    sd: float = 0.1, seed: int = 7, lattice_h: float = 2e-5,
                    nz: Optional[int] = None) -> Case:
    """A CuBe plate (Bonora damage) stretched in its plane at the strain rate
    `rate`, u = rate (x, y) (and u_z = 0 in 3D, nz cells thick, periodic in
    z), with a void material beside it (no void yet) and the yield stress
    perturbed by phi0 ~ rectified N(1, sd^2) on a lattice of spacing
    lattice_h; transmissive in x and y.  The stretch yields the plate, damage
    grows where the perturbed strength is low, and the void opens along the
    cracks that join them (Sec. 3.1): a state the step itself fractures, as
    in the expanding-disk and ring tests of Sec. 4.2 and 4.3.  The plate is
    L wide (n cells); at 64 cells on 1 mm the first cracks open within about
    200 steps, and the steps to fracture grow with n at a fixed L."""
    mats = [void(), cube("bonora")]
    dx = L / n
    half = 0.5 * L
    nz_ = (nz if nz is not None else 4) if dim == 3 else 1
    hz = 0.5 * nz_ * dx
    bc = [BC_TRANSMISSIVE] * 4 + ([BC_PERIODIC] * 2 if dim == 3 else [])
    case = Case("expanding_plate", dim, [n, n, nz_], [-half, -half, -hz if dim == 3 else 0],
                [half, half, hz if dim == 3 else 1], bc, mats, None, cfl=0.6, steps=300)
    lay = case.layout
    case.prim = blank_prim(lay, case.ncell)
    cen = case.centres()
    case.prim[lay.o_phi] = 0.0
    case.prim[lay.o_rho] = 0.0
    case.prim[lay.o_rho + 1] = mats[1]["rho0"]
    case.prim[lay.o_u] = rate * cen[0]
    case.prim[lay.o_u + 1] = rate * cen[1]
    case.prim[lay.o_p] = 1.0e5
    for d in range(dim):
        case.prim[lay.o_X + d] = cen[d]
    m = int(np.ceil(L / lattice_h)) + 3
    ext = half + lattice_h
    if dim == 2:
        case.phi0 = perturbation_gaussian(seed, [m, m], sd)
        case.pn, case.plo, case.ph = [m, m, 1], [-ext, -ext, 0], [lattice_h, lattice_h, 1]
    else:
        mz = int(np.ceil(2 * hz / lattice_h)) + 3
        case.phi0 = perturbation_gaussian(seed, [m, m, mz], sd)
        case.pn, case.plo = [m, m, mz], [-ext, -ext, -hz - lattice_h]
        case.ph = [lattice_h] * 3
    return case


def fractured_ring(n: int = 512, cracks: int = 12, seed: int = 11, **kw) -> Case:
    """The expanding-ring geometry at fragmentation (Sec. 4.3), input for
    fragment labelling: the annulus cut by `cracks` radial cracks of
    critically damaged metal (D = D_crit, as the RK4 cap leaves it) at
    stratified seeded angles, 1.5 cells wide; D ~ U(0, 0.9 D_crit) elsewhere.
    Solid fractions from 5 x 5 sub-sampling are multiples of 1/25, so no cell
    lies on a cut-off of 0.25, 0.5 or 0.75."""
    case = ring_2d(n, seed=seed, **kw)
    lay = case.layout
    r0, r1 = kw.get("r0", 0.020), kw.get("r1", 0.024)
    x, y = case.centres()
    dx = case.dx[0]
    case.prim[lay.o_phi] = np.clip(_annulus_fraction(x, y, dx, r0, r1, 5), PHI_MIN, 1.0 - PHI_MIN)
    Dc = case.materials[0]["D_crit"]
    crack = _crack_mask(case, np.hypot(x, y), np.arctan2(y, x),
                        2.0 * np.pi * _stratified(seed, cracks), np.zeros(0), None, 0.75 * dx)
    case.prim[lay.o_hist + 1] = np.where(crack, Dc, 0.9 * Dc * uniform01(seed + 1, case.ncell))
    return case


def fractured_cylinder(n: int = 256, cracks_theta: int = 8, cracks_z: int = 3, seed: int = 13,
                       nz: Optional[int] = None, **kw) -> Case:
    """The thin-cylinder geometry at fragmentation, input for fragment
    labelling: the shell cut by `cracks_theta` axial and `cracks_z`
    circumferential cracks of critically damaged metal (D = D_crit) at
    stratified seeded positions, 1.5 cells wide, periodic in z, so that it
    falls into cracks_theta x cracks_z patches; D ~ U(0, 0.9 D_crit)
    elsewhere; solid fractions from 5 x 5 sub-sampling (multiples of 1/25)."""
    case = cylinder_3d(n, seed=seed, nz=nz, **kw)
    lay = case.layout
    r0, r1 = kw.get("r0", 0.018), kw.get("r1", 0.020)
    x, y, z = case.centres()
    dx = case.dx[0]
    case.prim[lay.o_phi] = np.clip(_annulus_fraction(x, y, dx, r0, r1, 5), PHI_MIN, 1.0 - PHI_MIN)
    Dc = case.materials[0]["D_crit"]
    zc = case.lo[2] + (case.hi[2] - case.lo[2]) * _stratified(seed + 2, cracks_z)
    crack = _crack_mask(case, np.hypot(x, y), np.arctan2(y, x),
                        2.0 * np.pi * _stratified(seed, cracks_theta), zc, z, 0.75 * dx)
    case.prim[lay.o_hist + 1] = np.where(crack, Dc, 0.9 * Dc * uniform01(seed + 1, case.ncell))
    return case


WORKLOADS = {"spall_1d": spall_1d, "ring_2d": ring_2d, "cylinder_3d": cylinder_3d}
