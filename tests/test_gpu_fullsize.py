"""Parity at the full workload sizes in the launch configuration bench.py
times (512 x 512 ring, 256^3 cylinder): one GPU step of the whole grid,
checked on seeded sample cells that the oracle evaluates one by one from the
same initial state with the oracle's own full-grid CFL time step."""
import numpy as np
import pytest

from paper_2210_04037_gb300 import mmfrac, workloads as W
import subbox

pytestmark = pytest.mark.gpu

FULL = {"ring_2d_512": lambda: W.ring_2d(512), "cylinder_3d_256": lambda: W.cylinder_3d(256)}


@pytest.mark.parametrize("precision,tol", [(mmfrac.FP64, 1e-10), (mmfrac.FP32_SPLIT, 1e-3)])
@pytest.mark.parametrize("name", list(FULL))
def test_full_size_one_step_on_sampled_cells(name, precision, tol):
    case = FULL[name]()
    g = mmfrac.Grid(case, precision)
    info = g.step(1)
    out = g.read()
    g.close()
    dt, smax = subbox.oracle_cfl_dt(case)
    assert info["dt_last"] == pytest.approx(dt, rel=1e-12 if precision == mmfrac.FP64 else 1e-6)
    cells = subbox.sample_cells(case, 48, seed=11)
    assert len(cells) >= 30
    ref = np.stack([subbox.one_step_at(case, c, dt) for c in cells], axis=1)
    got = out[:, cells]
    num = np.abs(got - ref).sum(axis=1)
    den = np.abs(ref).sum(axis=1)
    rel = np.where(den > 0, num / np.where(den > 0, den, 1.0), num)
    names = case.layout.names()
    k = int(np.argmax(rel))
    assert rel.max() <= tol, f"{names[k]}: rel L1 over samples {rel[k]:.3e}"
