"""Batched and served FP64 runs against the FP64 CPU oracle directly (not
only against the same grid stepped alone on the GPU): every batch member and
every served run ends within 1e-10 relative L1 per field of the oracle after
the same number of steps, at the same time to 1e-12."""
import time

import numpy as np
import pytest

from oracle import OracleGrid
from paper_2210_04037_gb300 import mmfrac, workloads as W

pytestmark = pytest.mark.gpu


def rel_l1(out, ref):
    num = np.abs(out - ref).sum(axis=1)
    den = np.abs(ref).sum(axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def oracle_run(case, steps):
    o = OracleGrid(case)
    info = o.step(steps)
    return o.read(), info


def check(case, out, t, steps):
    ref, oinfo = oracle_run(case, steps)
    r = rel_l1(out, ref)
    names = case.layout.names()
    k = int(np.argmax(r))
    assert r.max() <= 1e-10, f"{case.name} {case.n}: {names[k]} rel L1 {r[k]:.3e}"
    assert t == pytest.approx(oinfo["t"], rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_fp64_batch_members_match_oracle(dim):
    if dim == 2:
        members, steps = [W.ring_2d(40, seed=10), W.ring_2d(56, seed=11)], 20
    else:
        members, steps = [W.cylinder_3d(n, nz=10, width=0.048, seed=40 + n) for n in (20, 24)], 10
    grids = [mmfrac.Grid(c, mmfrac.FP64) for c in members]
    b = mmfrac.Batch(grids)
    b.step(steps)
    outs = [(g.read(), g.synchronize()) for g in grids]
    b.close()
    for g in grids:
        g.close()
    for c, (out, info) in zip(members, outs):
        assert info["steps"] == steps
        check(c, out, info["t"], steps)


def test_fp64_served_runs_match_oracle():
    runs = [(W.ring_2d(40, seed=3), 12), (W.spall_1d(300), 30),
            (W.cylinder_3d(16, nz=10, width=0.048, seed=5), 5)]
    late = [(W.ring_2d(32, seed=7), 9), (W.spall_1d(200), 17)]
    srv = mmfrac.Server(steps_per_tick=4)
    ids = [srv.submit(c, n, precision=mmfrac.FP64) for c, n in runs]
    time.sleep(0.02)  # the later runs join while the first ones are stepping
    ids += [srv.submit(c, n, precision=mmfrac.FP64) for c, n in late]
    for rid, (case, n) in zip(ids, runs + late):
        info, out = srv.wait(rid, timeout=300)
        assert info["status"] == mmfrac.MM_OK and info["steps_done"] == n
        check(case, out, info["t"], n)
    srv.close()
