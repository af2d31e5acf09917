"""Long runs of the bench workloads stay admissible: the 512^2 ring for 500
steps in both precisions and the 128^3 cylinder for 300 FP32-split steps
(about ten times the bench horizon; without the half step's phase-density
bound, FP32-split runs of rings of this family stopped within about 100
steps at trace-fraction cells).  Every step's state passes the recovery's
checks or the run raises; the totals stay finite and the solid mass stays
within what the transmissive faces can have let out."""
import numpy as np
import pytest

from paper_2210_04037_gb300 import mmfrac, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [mmfrac.FP32_SPLIT, mmfrac.FP64])
def test_ring_512_runs_500_steps(prec):
    g = mmfrac.Grid(W.ring_2d(512), prec)
    T0 = g.totals()
    info = g.step(500)
    T1 = g.totals()
    g.close()
    assert info["steps"] == 500 and info["t"] > 0
    assert np.all(np.isfinite(T1))
    # the solid stays inside the box; trace outflow and FP32 rounding stay far below 1e-5
    assert abs(T1[0] - T0[0]) <= 1e-5 * T0[0]


def test_cylinder_128_runs_300_steps():
    g = mmfrac.Grid(W.cylinder_3d(128), mmfrac.FP32_SPLIT)
    T0 = g.totals()
    info = g.step(300)
    T1 = g.totals()
    g.close()
    assert info["steps"] == 300
    assert np.all(np.isfinite(T1))
    assert abs(T1[0] - T0[0]) <= 1e-5 * T0[0]
