"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point include/mmfrac.h declares; without a GPU it fails
loudly instead of falling back."""
import os
import re

import pytest

from paper_2210_04037_gb300 import mmfrac, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mm_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_entry_point():
    lib = mmfrac.load()
    names = declared()
    assert "mm_step" in names and "mm_create_grid" in names
    for n in names:
        assert hasattr(lib, n), n


def test_no_silent_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.Grid(W.spall_1d(32))
    assert e.value.status == mmfrac.MM_ECUDA


def test_invalid_descriptions_are_rejected_before_touching_a_device():
    c = W.spall_1d(32)
    c.n = [1, 1, 1]
    with pytest.raises(mmfrac.MMError) as e:
        mmfrac.create_grid(c)
    assert e.value.status == mmfrac.MM_EINVAL
