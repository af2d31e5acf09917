"""Build the CUDA library libmmfrac.so in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel with one -gencode; the FP64
units are compiled with --fmad=false (separate rounding of products and sums,
like the CPU reference arithmetic).  The FP32-split units take FP32 division
and square root to within 2 ulp (--prec-div=false --prec-sqrt=false, no IEEE
round-to-nearest sequences) and flush FP32 denormals (--ftz=true); their FP64
arithmetic (total energy, plastic-return iteration, totals) is unaffected.
Outputs land next to this file and are git-ignored.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmmfrac.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {"mm_api.cu": [], "mm_noalloc.cu": [], "mm_server.cu": [], "mm_frag.cu": []}
for _d in (1, 2, 3):
    for _b in ("", "_batch", "_void"):
        UNITS[f"mm_fp64_d{_d}{_b}.cu"] = ["--fmad=false"]
        UNITS[f"mm_fp32_d{_d}{_b}.cu"] = ["--prec-div=false", "--prec-sqrt=false", "--ftz=true"]
UNITS["mm_fp32_d3_tma.cu"] = UNITS["mm_fp32_d3.cu"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmmfrac")


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INC, "mmfrac.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra=(), out: str = LIB,
          build_dir: str = BUILD) -> str:
    if not force and out == LIB and up_to_date():
        return LIB
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
              *ARCH, *extra]

    def one(item):
        src, flags = item
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [cc, *common, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS.items()))
    tmp = out + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    t = build(force="--force" in sys.argv, verbose=True,
              extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(t)
