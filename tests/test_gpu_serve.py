"""Served runs with continuous batching through the C ABI: a run's result is
the same as the same grid stepped alone, whatever was served beside it (FP32-
split: to 1e-4 relative L1 per field, since the batched and single-grid
kernels may differ in FMA contraction; the momentum components and the
off-diagonal Fbar components against the L1 norm of their group, as in the
batch tests: the cylinder's axial momentum is 1e-3 of the total and grows
from rounding in the chaotic diffuse zone); admission follows the memory
budget; bounded waits time out."""
import time

import numpy as np
import pytest

from paper_2210_04037_gb300 import mmfrac, workloads as W

pytestmark = pytest.mark.gpu


def same_state(u, ref, lay):
    num = np.abs(u - ref).sum(axis=1)
    den = np.abs(ref).sum(axis=1)
    mom = list(range(lay.o_u, lay.o_u + lay.dim))
    off = [lay.F_index(i, j) for i in range(3) for j in range(3)
           if i != j and lay.F_index(i, j) is not None]
    for group in (mom, off):
        if group:
            den[group] = den[group].sum()
    r = num / np.where(den > 0, den, 1.0)
    k = int(np.argmax(r))
    return bool(r[k] <= 1e-4), f"{lay.names()[k]}: {r[k]:.3e}"


def alone(case, steps, prec=mmfrac.FP32_SPLIT):
    g = mmfrac.Grid(case, prec)
    info = g.step(steps)
    out = g.read()
    g.close()
    return out, info


def test_served_mix_equals_runs_alone():
    runs = [(W.ring_2d(48, seed=3), 12), (W.spall_1d(300), 30),
            (W.cylinder_3d(16, nz=10, width=0.048, seed=5), 5)]
    late = [(W.ring_2d(40, seed=7), 9), (W.spall_1d(200), 17),
            (W.cylinder_3d(18, nz=8, width=0.048, seed=6), 6)]
    srv = mmfrac.Server(steps_per_tick=4)
    ids = [srv.submit(c, n) for c, n in runs]
    time.sleep(0.02)  # the later runs arrive while the first ones are on the GPU
    ids += [srv.submit(c, n) for c, n in late]
    for rid, (case, n) in zip(ids, runs + late):
        info, out = srv.wait(rid, timeout=120)
        ref, rinfo = alone(case, n)
        assert info["status"] == mmfrac.MM_OK
        assert info["steps_done"] == n
        assert info["t"] == pytest.approx(rinfo["t"], rel=1e-6)
        assert info["submit_s"] <= info["admit_s"] <= info["done_s"]
        ok, worst = same_state(out, ref, case.layout)
        assert ok, (case.name, worst)
    st = srv.stats()
    assert st["used_bytes"] == 0 and st["pending"] == 0
    assert st["admitted"] == st["retired"] == len(ids)
    srv.close()


def test_memory_budget_serves_one_run_at_a_time():
    cases = [W.ring_2d(40, seed=11), W.ring_2d(40, seed=12), W.ring_2d(40, seed=13)]
    srv = mmfrac.Server(memory_budget=2_000_000, steps_per_tick=4)
    ids = [srv.submit(c, 8) for c in cases]
    infos = []
    for rid, case in zip(ids, cases):
        info, out = srv.wait(rid, timeout=120)
        infos.append(info)
        ok, worst = same_state(out, alone(case, 8)[0], case.layout)
        assert ok, (case.name, worst)
    for a, b in zip(infos, infos[1:]):
        assert b["admit_s"] >= a["done_s"]
    with pytest.raises(mmfrac.MMError) as e:
        srv.submit(W.ring_2d(256), 4)
    assert e.value.status == mmfrac.MM_EINVAL
    srv.close()


def test_bounded_wait_times_out_then_completes():
    srv = mmfrac.Server(steps_per_tick=2)
    case = W.ring_2d(96, seed=21)
    rid = srv.submit(case, 200)
    with pytest.raises(mmfrac.MMError) as e:
        srv.wait(rid, timeout=0)
    assert e.value.status == mmfrac.MM_ETIMEOUT
    info, out = srv.wait(rid, timeout=300)
    assert info["steps_done"] == 200
    with pytest.raises(mmfrac.MMError) as e:
        srv.wait(rid, timeout=0)  # already collected
    assert e.value.status == mmfrac.MM_EINVAL
    srv.close()


def test_submit_argument_errors():
    srv = mmfrac.Server()
    with pytest.raises(mmfrac.MMError) as e:
        srv.submit(W.ring_2d(32), -1)
    assert e.value.status == mmfrac.MM_EINVAL
    with pytest.raises(mmfrac.MMError) as e:
        srv.submit(W.ring_2d(32), 4, cfl=0.0)
    assert e.value.status == mmfrac.MM_EINVAL
    srv.close()
