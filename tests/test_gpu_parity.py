"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs, field by field.  FP64: relative L1 <= 1e-10 per
field (the arithmetic agrees up to libm ulps; see the design notes for the
bound).  FP32-split: relative L1 <= 1e-3 per field on smooth problems and
conserved totals within 1e-6."""
import numpy as np
import pytest

import cases
from oracle import OracleGrid
from paper_2210_04037_gb300 import mmfrac, workloads as W

pytestmark = pytest.mark.gpu


def rel_l1(out, ref):
    num = np.abs(out - ref).sum(axis=1)
    den = np.abs(ref).sum(axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def run_both(case, steps, precision=mmfrac.FP64):
    g = mmfrac.Grid(case, precision)
    G0 = g.totals()
    info = g.step(steps)
    out = g.read()
    tot = g.totals()
    g.close()
    o = OracleGrid(case)
    T0 = o.totals()
    oinfo = o.step(steps)
    return out, info, tot, o.read(), oinfo, o.totals(), T0, G0


# (case, steps).  100 steps wherever the dynamics are well posed; the ring and
# cylinder workloads at these coarse sizes are chaotic in their diffuse zones
# (the oracle against itself, with the initial state perturbed by 1e-15,
# diverges by 1e-9..1e-1 within 30-100 steps), so they run over the horizon
# on which two correct implementations still agree.
PARITY_CASES = {
    # spall workload at its full size (1000 cells, ragged against 64-cell tiles)
    "spall_1d_1000": (lambda: W.spall_1d(1000), 100),
    "ring_2d_90": (lambda: W.ring_2d(90), 60),
    "cylinder_3d_28x28x20": (lambda: W.cylinder_3d(28, nz=20, width=0.048), 30),
    # the largest sizes the oracle steps within a test's budget, over the
    # horizon on which the oracle started from a 1e-15 perturbation of the
    # same state still agrees with itself to 1e-10 (256^2: 3.3e-11 at 40
    # steps, 1.3e-4 at 60; 64^3: 3.8e-11 at 30, 6.6e-10 at 40)
    "ring_2d_256": (lambda: W.ring_2d(256), 40),
    "cylinder_3d_64": (lambda: W.cylinder_3d(64), 30),
    "periodic_mix_2d_50": (lambda: cases.periodic_mix_2d(50, shear=0.03), 100),
    "reflective_mix_2d_36": (lambda: cases.periodic_mix_2d(36, shear=0.03, bc=2), 100),
    "periodic_mix_3d_18x20x14": (lambda: cases.periodic_mix_3d(18, nz=14), 100),
    "reflective_mix_3d_12x14x10": (lambda: cases.periodic_mix_3d(12, nz=10, bc=2), 100),
    "sod_gas_1d_300": (lambda: cases.gas_riemann(300, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)), 100),
    "impact_al_periodic_1d": (lambda: cases.periodic_impact_1d(200), 100),
    # large enough that the 3D y and z sweeps run chunks of 9 consecutive
    # tiles per CTA, reusing each tile's overlap with the next
    "cylinder_3d_128_tile_chunks": (lambda: W.cylinder_3d(128), 3),
    # shear waves across a CuBe / Al-H32 interface moving at 2 m/s (the
    # oracle pin's case, boosted so that the normal velocity is not a
    # second-order field measured against its own tiny norm)
    "shear_bimaterial_2d": (lambda: _pin_shear_bimaterial(), 100),
    # reflective walls at both ends of one axis, the others periodic
    "reflective_walls_gas_1d": (lambda: _pin_reflective("gas_1d"), 60),
    "reflective_walls_solid_1d": (lambda: _pin_reflective("solid_1d"), 100),
    "reflective_walls_x_2d": (lambda: _pin_reflective("mix_2d_x"), 60),
    "reflective_walls_y_2d": (lambda: _pin_reflective("mix_2d_y"), 60),
    "reflective_walls_z_3d": (lambda: _pin_reflective("mix_3d_z"), 40),
    # the 2D mixture with shear laid in the y-z plane of a 3D grid (two
    # cells along x): the z sweep carries the in-plane shear
    "mix_2d_in_yz_plane_3d": (lambda: cases.embed_3d(cases.periodic_mix_2d(14, seed=3, shear=0.03),
                                                     (1, 2))[0], 60),
    # U-Nb with the Steinberg shear modulus and density-dependent Gamma
    # (R36): the compressed periodic mixture with yielding shear, and the
    # U-Nb ring of the expanding-ring test over its horizon (the oracle
    # against itself from a 1e-15 perturbation: 6e-11 at 20 steps)
    "steinberg_mix_2d_50": (lambda: cases.periodic_mix_2d(50, shear=0.03, solid=W.u_nb("simple")),
                            100),
    "steinberg_ring_unb_2d_256": (lambda: W.ring_unb_2d(256), 20),
}


def _pin_shear_bimaterial():
    import pins_waves as P
    L = 4e-3
    return cases.shear_bar_2d(600, L, lambda x: np.where(x < L / 2, -4.0, 12.0), left=P.CUBE,
                              right=P.AL, x0=L / 2, ux=2.0)


def _pin_reflective(kind):
    import pins_waves as P
    return P.reflective_case(kind)[0]


@pytest.mark.parametrize("name", list(PARITY_CASES))
def test_fp64_matches_oracle(name):
    make, steps = PARITY_CASES[name]
    case = make()
    out, info, tot, ref, oinfo, otot, _, _ = run_both(case, steps)
    r = rel_l1(out, ref)
    names = case.layout.names()
    worst = int(np.argmax(r))
    assert r.max() <= 1e-10, f"{names[worst]}: rel L1 {r[worst]:.3e}"
    assert info["steps"] == steps
    assert info["t"] == pytest.approx(oinfo["t"], rel=1e-12)
    assert np.allclose(tot, otot, rtol=1e-12, atol=1e-12 * np.abs(otot).max())


@pytest.mark.parametrize("name,make,steps", [
    ("spall_al_cube_1d_1000", lambda: W.spall_al_cube_1d(1000), 200),
    ("three_mix_2d_40", lambda: cases.three_mix_2d(40), 100),
])
def test_two_plastic_materials_fp64_matches_oracle(name, make, steps):
    """Three materials with two plastic solids (Sec. 4.1: the Al 5083 H32
    flyer onto the CuBe target in air; a smooth 2D Al/CuBe/air mixture with
    yielding shear): FP64 against the oracle to 1e-10 per conserved field
    and per primitive field but the phase densities.  A trace phase's
    density is the ratio of two trace quantities (1e-6 of air in the
    solids): the oracle against itself from a 1e-15 perturbation differs
    there by 4e-11 after 10 steps, while its conserved fields agree to
    1.5e-12 over 200 steps."""
    case = make()
    g = mmfrac.Grid(case, mmfrac.FP64)
    g.step(steps)
    U, w = g.read(False), g.read()
    tot = g.totals()
    g.close()
    o = OracleGrid(case)
    o.step(steps)
    Uo, wo = o.read(False), o.read()
    lay = case.layout
    r = rel_l1(U, Uo)
    k = int(np.argmax(r))
    assert r.max() <= 1e-10, f"{lay.cons_names()[k]}: rel L1 {r[k]:.3e}"
    rp = rel_l1(w, wo)
    rp[lay.o_rho:lay.o_rho + len(case.materials)] = 0.0
    k = int(np.argmax(rp))
    assert rp.max() <= 1e-10, f"{lay.names()[k]}: rel L1 {rp[k]:.3e}"
    assert np.allclose(tot, o.totals(), rtol=1e-12, atol=1e-12 * np.abs(o.totals()).max())


def test_two_plastic_materials_fp32_split_and_limits():
    """FP32-split on the three-material spall within 1e-3 of the oracle per
    conserved field (100 steps); two plastic materials are refused in 3D,
    with void, in batches and on the server."""
    case = W.spall_al_cube_1d(1000)
    g = mmfrac.Grid(case, mmfrac.FP32_SPLIT)
    g.step(100)
    U = g.read(False)
    g.close()
    o = OracleGrid(case)
    o.step(100)
    r = rel_l1(U, o.read(False))
    k = int(np.argmax(r))
    assert r.max() <= 1e-3, f"{case.layout.cons_names()[k]}: rel L1 {r[k]:.3e}"
    # 3D: not built for two plastic solids
    c3 = cases.embed_3d(cases.three_mix_2d(8), (0, 1))[0]
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.Grid(c3, mmfrac.FP64)
    assert e.value.status == mmfrac.MM_EINVAL
    # two plastic solids without a gas: single grids only
    two = W.Case("two", 2, [16, 16, 1], [0, 0, 0], [1e-3, 1e-3, 1], [1] * 4,
                 [W.al_h32("none"), W.cube("bonora")], None)
    lay = two.layout
    two.prim = W.blank_prim(lay, two.ncell)
    two.prim[lay.o_phi] = 0.5
    two.prim[lay.o_rho] = 2670.0
    two.prim[lay.o_rho + 1] = 8370.0
    two.prim[lay.o_p] = 1e5
    x, y = two.centres()
    two.prim[lay.o_X], two.prim[lay.o_X + 1] = x, y
    g2 = mmfrac.Grid(two, mmfrac.FP32_SPLIT)
    g2.step(3)
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.Batch([g2])
    assert e.value.status == mmfrac.MM_EINVAL
    g2.close()
    srv = mmfrac.Server(steps_per_tick=4)
    with pytest.raises(mmfrac.MMError):
        srv.submit(two, 4)
    srv.close()


def test_fp32_split_steinberg_against_oracle():
    """FP32-split with the Steinberg closure (R36) against the FP64 oracle
    on the smooth U-Nb/air mixture: relative L1 <= 1e-3 per field after 100
    steps."""
    case = cases.periodic_mix_2d(50, shear=0.01, vel=2.0, solid=W.u_nb("simple"))
    out, info, tot, ref, oinfo, otot, T0, G0 = run_both(case, 100, mmfrac.FP32_SPLIT)
    r = rel_l1(out, ref)
    names = case.layout.names()
    worst = int(np.argmax(r))
    assert r.max() <= 1e-3, f"{names[worst]}: rel L1 {r[worst]:.3e}"


def test_uniform_state_is_bitwise_preserved_on_gpu():
    n = 24
    c = W.Case("u", 2, [n, n, 1], [0, 0, 0], [1e-3, 1e-3, 1], [1, 1, 1, 1],
               [W.cube(), W.air()], None)
    lay = c.layout
    c.prim = W.blank_prim(lay, c.ncell)
    W.fill_two_phase(c, np.full(c.ncell, 0.7), 8000.0, 1.3, 2e8,
                     [np.full(c.ncell, 50.0), np.full(c.ncell, -20.0)])
    c.prim[lay.F_index(0, 1)] = 0.002
    for prec in (mmfrac.FP64, mmfrac.FP32_SPLIT):
        g = mmfrac.Grid(c, prec)
        U0 = g.read(False)
        g.step(20)
        U1 = g.read(False)
        g.close()
        for f in range(lay.o_X):
            assert np.array_equal(U1[f], U0[f]), (prec, lay.cons_names()[f])


def test_fp32_split_error_against_oracle_on_smooth_problem():
    case = cases.periodic_mix_2d(64, shear=0.01, vel=2.0)
    out, info, tot, ref, oinfo, otot, T0, G0 = run_both(case, 100, mmfrac.FP32_SPLIT)
    r = rel_l1(out, ref)
    names = case.layout.names()
    worst = int(np.argmax(r))
    assert r.max() <= 1e-3, f"{names[worst]}: rel L1 {r[worst]:.3e}"
    # conservation: the FP32-split run's totals against its own initial totals
    scale = np.abs(G0)
    mom = slice(2, 4)
    assert np.all(np.abs(tot[:2] - G0[:2]) <= 1e-6 * scale[:2])
    assert abs(tot[5] - G0[5]) <= 1e-6 * scale[5]
    assert np.all(np.abs(tot[mom] - G0[mom]) <= 1e-6 * max(1.0, np.abs(G0[mom]).max()) * 1e3)
    # representation of the initial state: the FP32 closure evaluates rho e
    # from terms (phi xi (p - p_ref), arho e_ref) up to ~10x the total energy
    # in this compressed mixture, each to FP32 rounding (6e-8): 1e-5 bounds it
    assert np.allclose(G0[:2], T0[:2], rtol=1e-7, atol=0)
    assert abs(G0[5] - T0[5]) <= 1e-5 * abs(T0[5])


@pytest.mark.parametrize("prec", [mmfrac.FP64, mmfrac.FP32_SPLIT])
def test_async_steps_equal_blocking_steps(prec):
    case = W.ring_2d(40)
    g1 = mmfrac.Grid(case, prec)
    i1 = g1.step(12)
    u1 = g1.read(False)
    g1.close()
    g2 = mmfrac.Grid(case, prec)
    for _ in range(3):
        g2.step_async(4)
    i2 = g2.synchronize()
    u2 = g2.read(False)
    g2.close()
    assert np.array_equal(u1, u2)
    assert i1 == i2


@pytest.mark.parametrize("prec", [mmfrac.FP64, mmfrac.FP32_SPLIT])
@pytest.mark.parametrize("make", [lambda: W.ring_2d(40), lambda: W.cylinder_3d(16, nz=8, width=0.048)])
def test_graph_replay_equals_launch_by_launch(prec, make):
    # per-launch timing forces launch-by-launch stepping; otherwise steps after
    # the first replay a captured step (two graphs in 3D, recaptured on a cfl change)
    case = make()
    out = []
    for timed in (True, False):
        g = mmfrac.Grid(case, prec)
        mmfrac.profile_enable(g.h, timed)
        g.step(5)
        g.step(3, cfl=0.4)
        g.step(2)
        out.append((g.read(False), g.synchronize()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_inadmissible_initial_state_is_reported():
    c = W.spall_1d(64)
    c.prim[c.layout.o_rho, 10] = -1.0
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.Grid(c)
    assert e.value.status == mmfrac.MM_ENONFINITE
    assert "cell 10" in str(e.value)


def test_argument_errors():
    c = W.spall_1d(64)
    g = mmfrac.Grid(c)
    with pytest.raises(mmfrac.MMError) as e:
        g.step(1, cfl=0.0)
    assert e.value.status == mmfrac.MM_EINVAL
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.read_fields(g.h, out=np.empty((1, 3)))
    assert e.value.status == mmfrac.MM_EINVAL
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.step_async(g.h, -1, 0.5)
    assert e.value.status == mmfrac.MM_EINVAL
    g.close()
    h = mmfrac.create_grid(c)
    for call in (lambda: mmfrac.step(h, 1, 0.5), lambda: mmfrac.step_async(h, 1, 0.5),
                 lambda: mmfrac.synchronize(h)):
        with pytest.raises(mmfrac.MMError) as e:
            call()
        assert e.value.status == mmfrac.MM_ESTATE
    mmfrac.destroy(h)
