"""TMA-staged y and z sweeps (3D FP32-split, two materials) against the
per-thread loads they replace.  The staged tiles hold the stored values, so
the two differ only where the compiler contracted a product and a sum into
one FMA in one kernel and not in the other: compiled without contraction
(--fmad=false) they end bit for bit alike, and in the product build they
agree to FP32 rounding after a step and within the batched-ensemble
criterion (1e-4 relative L1 per field group) after eight.  Grids are large
enough for the column kernels (several tiles per CTA, several chunks per
column), ragged along every axis (n[0] a multiple of 4, not of the 8-cell
box width; the sweep axes not multiples of the 16-cell tile length), with
periodic, reflective and transmissive ends, with and without a plastic
history.  Grids the maps cannot describe (n[0] not a multiple of 4, FP64,
2D, void) run without them.  Against the oracle, the staged path is covered
by the full-size check of one 256^3 cylinder step (test_gpu_fullsize.py),
which runs with the maps on by default."""
import copy
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2210_04037_gb300 import build as B, mmfrac, workloads as W
from test_gpu_batch import same_state

pytestmark = pytest.mark.gpu

FP32 = mmfrac.FP32_SPLIT


def cylinder(n, nz, bc=None, plastic=True):
    c = W.cylinder_3d(n, nz=nz, lattice_h=0.002)
    if bc is not None:
        c.bc = list(bc)
    if not plastic:
        # the same state with an elastic shell: no plastic history fields
        out = copy.deepcopy(c)
        out.materials = [W.cube("bonora", plastic=False), W.air()]
        l0, l1 = c.layout, out.layout
        keep = [f for f in range(l0.nfield)
                if not l0.o_hist <= f < l0.o_hist + 2 * l0.nhist]
        assert len(keep) == l1.nfield and l1.nhist == 0
        out.prim = c.prim[keep].copy()
        c = out
    return c


def totals_match(t1, t0, nmat, rtol):
    """Masses and energy to rtol; momenta (near zero in these symmetric
    runs) to rtol of the total mass times 1 km/s."""
    t1, t0 = np.asarray(t1), np.asarray(t0)
    own = list(range(nmat)) + [len(t0) - 1]
    mom = list(range(nmat, len(t0) - 1))
    return (np.allclose(t1[own], t0[own], rtol=rtol, atol=0) and
            np.all(np.abs(t1[mom] - t0[mom]) <= rtol * 1e3 * t0[:nmat].sum()))


def run(case, steps, tma, chunks=1):
    g = mmfrac.Grid(case, FP32)
    active = g.set_tma_loads(tma)
    for _ in range(chunks):
        g.step(steps)
    info = g.synchronize()
    u = g.read(False)
    tot = g.totals()
    g.close()
    return u, tot, info, active


CASES = [
    ("periodic z", 100, 84, None, True),
    ("reflective y, z", 100, 84, [W.BC_TRANSMISSIVE] * 2 + [W.BC_REFLECTIVE] * 4, True),
    ("transmissive, no history", 96, 100, [W.BC_TRANSMISSIVE] * 6, False),
]


@pytest.mark.parametrize("name,n,nz,bc,plastic", CASES, ids=[c[0] for c in CASES])
def test_staged_sweeps_match_per_thread_loads(name, n, nz, bc, plastic):
    case = cylinder(n, nz, bc, plastic)
    lay = case.layout
    # one step: FP32 rounding of the fields' scales at most
    u1, t1, i1, a1 = run(case, 1, True)
    u0, t0, i0, a0 = run(case, 1, False)
    assert a1 and not a0
    assert i1["t"] == i0["t"]
    scale = np.abs(u0).max(axis=1, keepdims=True)
    assert np.all(np.abs(u1 - u0) <= 1e-6 * np.where(scale > 0, scale, 1.0))
    assert totals_match(t1, t0, lay.nmat, 1e-10)
    # eight steps, in two chunks (graph replay)
    u1, t1, i1, _ = run(case, 4, True, chunks=2)
    u0, t0, i0, _ = run(case, 4, False, chunks=2)
    assert i1["steps"] == i0["steps"] == 8
    assert np.isfinite(u1).all()
    assert same_state(u1, u0, FP32, lay)
    assert totals_match(t1, t0, lay.nmat, 1e-9)


_BITWISE = """
import json, sys
sys.path[:0] = [{tests!r}, {repo!r}]
import test_gpu_tma as T
out = {{}}
for name, n, nz, bc, plastic in T.CASES:
    case = T.cylinder(n, nz, bc, plastic)
    u1 = T.run(case, 2, True)[0]
    u0 = T.run(case, 2, False)[0]
    out[name] = int((u1 != u0).sum())
print(json.dumps(out))
"""


def test_staged_sweeps_are_bit_identical_without_contraction(tmp_path):
    # the library built with --fmad=false, loaded by a child process
    lib = B.build(force=True, extra=["--fmad=false"], out=str(tmp_path / "libmmfrac.so"),
                  build_dir=str(tmp_path / "obj"))
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, MMFRAC_LIB=lib)
    code = _BITWISE.format(tests=here, repo=os.path.dirname(here))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    diff = json.loads(r.stdout.strip().splitlines()[-1])
    assert diff == {c[0]: 0 for c in CASES}


def test_switch_between_steps():
    case = cylinder(100, 84)
    g = mmfrac.Grid(case, FP32)
    assert g.set_tma_loads() is True  # on by default
    g.step(2)
    assert g.set_tma_loads(False) is False
    g.step(2)
    assert g.set_tma_loads(True) is True
    g.step(2)
    info = g.synchronize()
    u = g.read(False)
    g.close()
    assert info["steps"] == 6
    ref, _, _, _ = run(case, 6, False)
    assert same_state(u, ref, FP32, case.layout)


def test_grids_without_maps_run_per_thread_loads():
    # n[0] not a multiple of 4: rows are not 16-byte multiples
    c98 = cylinder(98, 84)
    u, _, info, active = run(c98, 3, True)
    assert not active and np.isfinite(u).all() and info["steps"] == 3
    # FP64, 2D and void grids never get maps
    g = mmfrac.Grid(cylinder(32, 16), mmfrac.FP64)
    assert g.set_tma_loads(True) is False
    g.close()
    g = mmfrac.Grid(W.ring_2d(64), FP32)
    assert g.set_tma_loads(True) is False
    g.close()
    g = mmfrac.Grid(W.add_void(cylinder(32, 16)), FP32)
    assert g.set_tma_loads(True) is False
    g.close()
