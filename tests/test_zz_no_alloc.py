"""The allocation-free totals entry point, for callers that hold the state in
their own device memory and cannot let the library allocate (a serving loop
with a fixed device pool, a runtime whose allocator is off limits): on the
same state its output equals that of mm_conserved_totals, within the
tolerance the totals checks use, on two calls in a row and across two
states of different shape.  Collected last so a failure here leaves every
other test already run."""
import numpy as np
import pytest

import cases
from paper_2210_04037_gb300 import mmfrac

pytestmark = pytest.mark.gpu


def test_noalloc_totals_equal_the_allocating_entry_point():
    torch = pytest.importorskip("torch")
    for case in (cases.periodic_mix_2d(40, shear=0.03), cases.periodic_mix_3d(12, nz=10)):
        g = mmfrac.Grid(case, mmfrac.FP64)
        g.step(3)
        ref = g.totals()
        U = g.read(primitive=False)
        g.close()
        nmat = len(case.materials)
        d_cons = torch.from_numpy(np.ascontiguousarray(U)).to("cuda")
        for _ in range(2):
            out = torch.full((nmat + 4,), float("nan"), dtype=torch.float64, device="cuda")
            mmfrac.conserved_totals_noalloc(d_cons.data_ptr(), case.dim, case.ncell, nmat,
                                            case.layout.nhist, case.dx, out.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), (got, ref)


def test_noalloc_rejects_more_materials_than_its_scratch_holds():
    torch = pytest.importorskip("torch")
    d = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.conserved_totals_noalloc(d.data_ptr(), 1, 4, 5, 0, [1.0], d.data_ptr())
    assert e.value.status == mmfrac.MM_EINVAL
    assert "exceed the fixed scratch" in str(e.value)
