"""The allocation-free totals entry point, for callers that hold the state in
their own device memory and cannot let the library allocate (a serving loop
with a fixed device pool, a runtime whose allocator is off limits): on the
same state its output equals that of mm_conserved_totals, within the
tolerance the totals checks use, on two calls in a row and across states of
different shape (1D, 2D, 3D; one, two and three materials), and calls after
the first leave the device's free memory unchanged.  Collected last so a
failure here leaves every other test already run."""
import numpy as np
import pytest

import cases
import pins_void as PV
from paper_2210_04037_gb300 import mmfrac

pytestmark = pytest.mark.gpu


def _states():
    yield cases.periodic_mix_2d(40, shear=0.03)
    yield cases.periodic_mix_3d(12, nz=10)
    yield cases.spall_like_1d(300)  # 1D: momenta 1, 2 are zero, dx padded
    yield cases.elastic_cube(200, 1e-3, lambda x: 5.0 * np.sin(2 * np.pi * x / 1e-3))  # one material
    yield PV.bar()  # void, CuBe: two materials, one plastic
    from paper_2210_04037_gb300 import workloads as W
    yield W.add_void(W.ring_2d(48, seed=3))  # three materials


def test_noalloc_totals_equal_the_allocating_entry_point():
    torch = pytest.importorskip("torch")
    for case in _states():
        g = mmfrac.Grid(case, mmfrac.FP64)
        g.step(3)
        ref = g.totals()
        U = g.read(primitive=False)
        g.close()
        nmat = len(case.materials)
        d_cons = torch.from_numpy(np.ascontiguousarray(U)).to("cuda")
        free = []
        for _ in range(3):
            out = torch.full((nmat + 4,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            before = torch.cuda.mem_get_info()[0]
            mmfrac.conserved_totals_noalloc(d_cons.data_ptr(), case.dim, case.ncell, nmat,
                                            case.layout.nhist, case.dx, out.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            free.append((before, torch.cuda.mem_get_info()[0]))
            got = out.cpu().numpy()
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), \
                (case.name, got, ref)
        # the first call in the process may load the device code; later
        # calls allocate nothing
        for b, a in free[1:]:
            assert a == b, (case.name, b, a)


def test_noalloc_rejects_more_materials_than_its_scratch_holds():
    torch = pytest.importorskip("torch")
    d = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.conserved_totals_noalloc(d.data_ptr(), 1, 4, 5, 0, [1.0], d.data_ptr())
    assert e.value.status == mmfrac.MM_EINVAL
    assert "exceed the fixed scratch" in str(e.value)
