"""Throughput of the explicit diffuse-interface step on GB300.

One step = CFL time step + the dimensionally split sweeps + the per-cell
sources, over the whole grid of the workload.  Metric: cell-updates/s (one
update = one cell through one full step), for the FP32-split path (the
headline) beside the FP64 path, with the HBM roofline fraction of the
dominant kernel.

    python bench.py [--gpus N --steps K --warmup W]
                    [--workload cylinder_3d|ring_2d|spall_1d|ensemble_2d|serve|fragments]
                    [--precision fp32split|fp64] [--impl mmfrac|reference]

``--workload ensemble_2d`` times a batch of seeded 2D rings of uneven size
(``--size`` members, default 64) stepped together, beside the same members
stepped one at a time in FP32-split and in FP64.  ``--workload fragments``
times the fragment labelling (cells labelled/s) of a fractured 3D shell
(``--size`` cells per edge, default 256), with its own metric.

With N > 1 (torchrun) every rank runs an independent replica of the
workload (the step does not shard on one grid here: replicas only); the
value is the aggregate over ranks.  ``--impl reference`` times the CPU
oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2210_04037_gb300 import workloads as W  # noqa: E402

METRIC = ("cell-updates/s and % HBM roofline at 1 GB300, FP32-split vs FP64 at stated error")
L2_BYTES = 129 * 2 ** 20
DEFAULT_SIZE = {"ring_2d": 512, "cylinder_3d": 256, "spall_1d": 1000, "ensemble_2d": 64,
                "serve": 24, "fragments": 256}
FRAG_METRIC = "fragment labelling at void cut-off 0.5: cells labelled/s at 1 GB300"
FRAG_CUT = 0.5
WORKLOAD_TEXT = {
    "ring_2d": "2D expanding ring, {n}x{n} cells, Al-H32 annulus r 20-24 mm at 200 m/s in air, "
               "simple damage, phi0 ~ U(0.9,1.1) on a 0.5 mm lattice",
    "cylinder_3d": "3D expanding thin cylinder, {n}^3 cells, CuBe shell r 18-20 mm at 250 m/s in "
                   "air, Bonora damage, phi0 ~ rectified N(1,0.1^2) on a 0.5 mm lattice",
    "spall_1d": "1D plate impact spall, {n} cells, CuBe flyer 2 mm at 300 m/s onto a 6 mm "
                "target, Bonora damage, phi0 ~ rectified N(1,0.05^2) per cell",
    "ensemble_2d": "batched ensemble: {n} seeded 2D expanding rings (the ring workload, seeds "
                   "100..), grids uneven 128^2..768^2 in steps of 8, stepped together: one launch "
                   "per kernel kind over all members, CUDA graph replay, autotuned tile shapes and persistent CTAs per SM",
    "serve": "served runs: {n} requests with Poisson arrivals (16/s, seeded) mixing 1D spall "
             "(1e3..1e4 cells, 400 steps), 2D ring (256^2..1024^2, 60 steps) and 3D cylinder "
             "(128^3..256^3, 10 steps), FP32-split, memory-based admission, continuous batching",
    "fragments": "fragment labelling (mm_fragments, void cut-off 0.5) of a 3D thin-cylinder shell "
                 "at fragmentation, {n}^3 cells: CuBe shell r 18-20 mm, periodic in z, cut by 12 "
                 "axial and 4 circumferential cracks 1.5 cells wide at D_crit (48 patches), "
                 "D ~ U(0, 0.9 D_crit) elsewhere",
}


def serve_requests(count: int, seed: int = 7, rate: float = 16.0):
    """(kind, size, steps, arrival time in s) of each request: seeded."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(count):
        kind = rng.choice(["1d", "2d", "3d"], p=[0.35, 0.45, 0.2])
        if kind == "1d":
            n, steps = int(rng.integers(1000, 10001)), 400
        elif kind == "2d":
            n, steps = int(rng.choice([256, 384, 512, 640, 768, 1024])), 60
        else:
            n, steps = int(rng.choice([128, 160, 192, 256], p=[0.4, 0.3, 0.2, 0.1])), 10
        out.append((str(kind), n, steps, t))
        t += float(rng.exponential(1.0 / rate))
    return out


def serve_case(kind: str, n: int, seed: int):
    if kind == "1d":
        return W.spall_1d(n)
    if kind == "2d":
        return W.ring_2d(n, seed=seed)
    return W.cylinder_3d(n, seed=seed)


def ensemble_sizes(m: int):
    """Grid edge of each member: 128 .. 768 evenly, multiples of 8."""
    return [128 + 8 * round(80 * i / max(m - 1, 1)) for i in range(m)]


def ensemble_cases(m: int):
    return [W.ring_2d(n, seed=100 + i) for i, n in enumerate(ensemble_sizes(m))]


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum, cold L2) per
# launch of the bench's kernels at their default size, with the SHA-256 of the
# kernel sources and build script they were measured on; reported as null
# once those differ.
TRAFFIC_SRC_SHA256 = "0647811e1ea81d79d230a83fbd06aa655f02c43780d0a568fc85f84576ba79c4"
TRAFFIC = {("cylinder_3d", 256, "fp32split"): {"sweep_x": 3041095168, "sweep_y": 3269300736,
                                               "sweep_z": 3333256192, "sources": 1816213504,
                                               "cfl": 1545776384}}


def kernel_src_hash() -> str:
    """SHA-256 of what the single-grid step kernels are built from: the
    kernel headers, the per-precision single-grid units and build.py (not
    the host API, the batch units or fragment labelling)."""
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2210_04037_gb300", "csrc")
    step = [f for f in sorted(os.listdir(cs))
            if f.endswith((".cuh", ".h")) or (f.startswith("mm_fp") and "_batch" not in f)]
    for f in step + ["../build.py"]:
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(workload: str, n: int, precision: str, kernel: str):
    t = TRAFFIC.get((workload, n, precision), {}).get(kernel)
    if t is None or kernel_src_hash() != TRAFFIC_SRC_SHA256:
        return None
    return t


def fragment_case(n: int):
    return W.fractured_cylinder(n, 12, 4, seed=6)


def frag_bytes_per_cell(precision: int, member_frac: float) -> dict:
    """Algorithmic DRAM bytes per cell of each labelling kernel kind.
    mark: the stored fractions (FP64: the N-1 stored ones; FP32-split: all
    N), the solid's phi rho and phi rho D read, a parent index (4 B) written,
    and a mass (8 B) on fragment cells.  union: parents read by the merge and
    read and written (members) by the root pass.  count: parents read.
    collect: parents read twice (numbering, sums) and the members' masses."""
    e = 8 if precision == W.FP64 else 4
    nfrac = 1 if precision == W.FP64 else 2
    return {"frag_mark": (nfrac + 2) * e + 4 + 8 * member_frac,
            "frag_union": 8 + 4 * member_frac,
            "frag_count": 4, "frag_collect": 8 + 8 * member_frac}


def make_case(name: str, n: int):
    if name == "fragments":
        return fragment_case(n)
    if name == "ensemble_2d":
        # the oracle's sample of an ensemble: its smallest member
        return ensemble_cases(n)[0]
    if name == "serve":
        # the oracle's sample of the served mix: its smallest 2D ring
        return W.ring_2d(256)
    return W.WORKLOADS[name](n)


def max_over_ranks(value: float, dist=None, device: str = "cuda") -> float:
    """Largest value over the ranks of the process group (the timing rule:
    the slowest replica sets the time); the value itself on one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(cells_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job cell-updates/s: every rank advances its own replica."""
    return world * cells_per_rank * steps / (ms_max * 1e-3)


def algo_bytes_per_pass(case, precision: int) -> int:
    """Algorithmic bytes per cell of one split pass: one read and one write
    of the S stored fields of the method's state (S = 21 in 3D, 15 in 2D, 11
    in 1D for two materials with one plastic one).  FP64: 8 bytes a field;
    FP32-split: rho E in 8 bytes and the other S - 1 fields in 4.  A full
    step moves `dim` times this.  The build's own layout (`state_bytes`)
    carries the last volume fraction too and is reported beside it."""
    s = case.layout.nfield
    return 2 * 8 * s if precision == W.FP64 else 2 * (8 + 4 * (s - 1))


def state_bytes(case, precision: int) -> int:
    """Bytes of one copy of the conserved state: FP64 stores every field in
    8 bytes; FP32-split stores rho E in 8 bytes and every other field, plus
    the carried last volume fraction, in 4."""
    nf = case.layout.nfield
    per = 8 * nf if precision == W.FP64 else 4 * nf + 8
    return per * case.ncell


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(case_name: str, n: int, budget_s: float = 12.0, max_steps: int = 50):
    """The FP64 CPU oracle as it stands, on the host cores, over a bounded
    number of steps of the same workload (the CPU reference)."""
    from oracle import OracleGrid
    case = make_case(case_name, n)
    cores = os.cpu_count() or 1
    g = OracleGrid(case, threads=cores)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (time.perf_counter() - t0) < budget_s:
        g.step(1)
        steps += 1
    el = time.perf_counter() - t0
    return {"value": case.ncell * steps / el, "unit": "cell-updates/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{steps} FP64 steps of the same {case.ncell}-cell workload"
                      + (" (the ensemble's smallest member)" if case_name == "ensemble_2d" else "")
                      + " from its "
                      f"initial state ({el:.1f} s wall)"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    n = args.size or DEFAULT_SIZE[args.workload]
    from oracle import OracleGrid
    case = make_case(args.workload, n)
    cores = os.cpu_count() or 1
    g = OracleGrid(case, threads=cores)
    if args.workload == "fragments":
        return run_reference_fragments(args, world, case, g, n)
    # a bounded sample: the warm-up and the timed steps each stop after about
    # a minute of host time (the 256^3 cylinder takes seconds per step)
    t0 = time.perf_counter()
    warm = 0
    while warm < args.warmup and (warm == 0 or time.perf_counter() - t0 < 30.0):
        g.step(1)
        warm += 1
    t0 = time.perf_counter()
    steps = 0
    while steps < args.steps and (steps == 0 or time.perf_counter() - t0 < 60.0):
        g.step(1)
        steps += 1
    el = time.perf_counter() - t0
    value = case.ncell * steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload].format(n=n), "cells": case.ncell,
                       "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{steps} timed FP64 steps of the full workload "
                                       f"after {warm} warm-up steps (at most {args.steps} and "
                                       f"{args.warmup}, each run capped near a minute)"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_fragments(args, world: int, case, g, n: int):
    """The oracle's labelling (single-threaded breadth-first search) of the
    full workload, as many calls as fit in about 20 s (at most --steps)."""
    g.fragments(FRAG_CUT)
    t0 = time.perf_counter()
    calls = 0
    while calls < max(1, args.steps) and (calls == 0 or time.perf_counter() - t0 < 20.0):
        g.fragments(FRAG_CUT)
        calls += 1
    el = time.perf_counter() - t0
    value = case.ncell * calls / el
    sample = f"{calls} labellings of the full {case.ncell}-cell workload after one untimed"
    line = {"impl": "reference", "metric": FRAG_METRIC, "value": value, "unit": "cells/s",
            "n_gpus": world, "steps": calls, "warmup": 1, "ms_per_step": 1e3 * el / calls,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["fragments"].format(n=n), "cells": case.ncell,
                       "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_fragments(args, rank: int, world: int):
    """Device time of mm_fragments calls on a resident fractured state, the
    per-kernel times, the end-to-end call from host buffers, and the
    oracle's labelling of the same state beside it."""
    import torch
    from paper_2210_04037_gb300 import mmfrac
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.size or DEFAULT_SIZE["fragments"]
    case = fragment_case(n)
    prec = W.FP32_SPLIT if args.precision == "fp32split" else W.FP64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sbytes = state_bytes(case, prec)
    flush = None
    if sbytes < 2 * L2_BYTES:
        flush = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    g = mmfrac.Grid(case, prec, stream=stream.cuda_stream)
    for _ in range(max(1, args.warmup)):
        lab, f = g.fragments(FRAG_CUT, labels=True, max_frags=0)
    member_frac = float((lab >= 0).mean())
    nfrag = f["n"]
    calls = args.steps
    start = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    stop = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = 0
    with ClockSampler(local) as clk:
        for s in range(calls):
            if flush is not None:
                flush.add_(1)
            l0 = g.launches()
            start[s].record(stream)
            g.fragments(FRAG_CUT, labels=False, max_frags=0)
            stop[s].record(stream)
            launches += g.launches() - l0
        torch.cuda.synchronize()
        # the same calls with events around each kernel kind
        mmfrac.profile_enable(g.h, True)
        mmfrac.profile_read(g.h, reset=True)
        for s in range(calls):
            if flush is not None:
                flush.add_(1)
            g.fragments(FRAG_CUT, labels=False, max_frags=0)
        prof = mmfrac.profile_read(g.h, reset=True)
        mmfrac.profile_enable(g.h, False)
        torch.cuda.synchronize()
    g.close()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(start, stop)), dist)
    value = world * case.ncell * calls / (ms * 1e-3)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    per_cell = frag_bytes_per_cell(prec, member_frac)
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms = kinds[dom][0] / kinds[dom][1]
    algo = per_cell[dom] * case.ncell
    peak, peak_kind = read_peaks()
    achieved = algo / (dom_ms * 1e-3) / 1e9
    # end to end: the state uploaded from pinned host memory, labelled, the
    # labels read back (4 B per cell from the device), the grid released
    prim_pinned = torch.from_numpy(np.ascontiguousarray(case.prim)).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(calls):
        h = mmfrac.create_grid(case, prec, stream.cuda_stream)
        mmfrac.set_materials(h, case, prim=prim_pinned.numpy())
        mmfrac.fragments(h, FRAG_CUT, labels=True, max_frags=nfrag)
        mmfrac.destroy(h)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    h2d = case.prim.nbytes + (case.phi0.nbytes if case.phi0 is not None else 0)
    d2h = 4 * case.ncell + 24 * nfrag + 4
    line = {
        "metric": FRAG_METRIC, "value": value, "unit": "cells/s", "n_gpus": world,
        "steps": calls, "warmup": args.warmup, "ms_per_step": ms / calls,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == W.FP32_SPLIT else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["fragments"].format(n=n), "cells": case.ncell,
                   "precision": args.precision, "fragments": nfrag,
                   "member_fraction": member_frac,
                   "l2": "flushed between calls (256 MiB write)" if flush is not None
                   else "state larger than L2",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": measured_traffic("fragments", n, args.precision, dom),
                     "algorithmic_bytes_per_launch": algo, "avg_launch_ms": dom_ms},
        "kernels_ms_per_call": {k: v[0] / calls for k, v in kinds.items()},
        "e2e": {"value": world * case.ncell * calls / e2e_s, "unit": "cells/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import OracleGrid
        o = OracleGrid(case)
        t0 = time.perf_counter()
        o.fragments(FRAG_CUT)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": case.ncell / el, "unit": "cells/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"one labelling of the full {case.ncell}-cell workload "
                                          f"({el:.1f} s wall, single-threaded search)"}
    if not args.no_extra:
        line["self_fractured"] = run_self_fractured(args, prec, stream, calls, dist, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


SELF_FRACTURED_N = 1024


def run_self_fractured(args, prec, stream, calls, dist, rank, world):
    """Fragment labelling on a state the step itself fractured: the
    expanding CuBe plate (workloads.expanding_plate, 1024^2, a void material
    beside it) stepped on the GPU until it has broken into fragments (not
    timed), then `calls` labellings timed with CUDA events, L2 flushed
    between them; the labels checked against the oracle's labelling of the
    same state."""
    import torch
    from paper_2210_04037_gb300 import mmfrac
    case = W.expanding_plate(SELF_FRACTURED_N)
    g = mmfrac.Grid(case, prec, stream=stream.cuda_stream)
    steps, nfrag = 0, 1
    while steps < 12000 and nfrag < 8:
        g.step(250)
        steps += 250
        nfrag = g.fragments(FRAG_CUT, labels=False, max_frags=0)[1]["n"]
    info = g.synchronize()
    lab, f = g.fragments(FRAG_CUT, labels=True, max_frags=0)
    flush = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    start = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    stop = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for s in range(calls):
        flush.add_(1)
        start[s].record(stream)
        g.fragments(FRAG_CUT, labels=False, max_frags=0)
        stop[s].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(start, stop)), dist)
    U = g.read(primitive=False)
    g.close()
    out = {"workload": f"CuBe plate 1 mm, {SELF_FRACTURED_N}^2 cells, stretched in-plane at "
                       f"2e5/s (workloads.expanding_plate), fractured by {steps} steps of its "
                       f"own ({args.precision}, t = {info['t'] * 1e6:.2f} us)",
           "cells": case.ncell, "steps_to_fracture": steps, "fragments": f["n"],
           "member_fraction": float((lab >= 0).mean()),
           "value": world * case.ncell * calls / (ms * 1e-3), "unit": "cells/s",
           "ms_per_call": ms / calls, "l2": "flushed between calls (256 MiB write)"}
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import OracleGrid
        o = OracleGrid(case)
        o.write_conserved(U)
        t0 = time.perf_counter()
        olab, of = o.fragments(FRAG_CUT)
        el = time.perf_counter() - t0
        # (the FP32-split state stores every volume fraction; the oracle forms
        # the last as 1 - sum, so a cell within FP32 rounding of the cut-off
        # can fall on the other side)
        out["oracle_fragments"] = of["n"]
        out["cells_labelled_differently_from_oracle"] = int((olab != lab).sum())
        out["cpu_baseline"] = {"value": case.ncell / el, "unit": "cells/s", "cores": 1,
                               "kind": "oracle", "sample": "one labelling of the same state"}
    return out


def time_device(case, precision, steps, warmup, stream, flush_buf, profile=True, x_transport=0):
    """Device time of `steps` single-step calls (CUDA events on the grid's
    stream), L2 flushed between steps when the state fits in L2."""
    import torch
    from paper_2210_04037_gb300 import mmfrac
    g = mmfrac.Grid(case, precision, stream=stream.cuda_stream, x_transport=x_transport)
    g.step(warmup)
    mmfrac.profile_enable(g.h, profile)
    mmfrac.profile_read(g.h, reset=True)
    start = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    stop = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches = 0
    torch.cuda.synchronize()
    for s in range(steps):
        if flush_buf is not None:
            flush_buf.add_(1)
        start[s].record(stream)
        g.step_async(1)
        stop[s].record(stream)
        launches += g.launches()
    g.synchronize()  # raises on a failure latched by any of the steps
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(start, stop))
    prof = mmfrac.profile_read(g.h, reset=True)
    return g, ms, prof, launches


def time_alone(cases, precision, steps, stream):
    """Each member alone (created, one warm-up step, `steps` timed enqueued
    steps, freed): summed device time."""
    import torch
    from paper_2210_04037_gb300 import mmfrac
    total = 0.0
    for c in cases:
        g = mmfrac.Grid(c, precision, stream=stream.cuda_stream)
        g.step(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step_async(steps)
        e1.record(stream)
        g.synchronize()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
        g.close()
    return total


def run_ensemble(args, rank: int, world: int, nested: bool = False, dist=None):
    """The batched ensemble's line; nested: inside another workload's run
    (process group and device already set up, nothing printed, the line
    returned)."""
    import torch
    from paper_2210_04037_gb300 import mmfrac
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1 and not nested:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    m = (args.size if not nested else 0) or DEFAULT_SIZE["ensemble_2d"]
    members = ensemble_cases(m)
    ncell = sum(c.ncell for c in members)
    prec = W.FP32_SPLIT if args.precision == "fp32split" else W.FP64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    grids = [mmfrac.Grid(c, prec, stream=stream.cuda_stream) for c in members]
    b = mmfrac.Batch(grids, stream=stream.cuda_stream)
    b.step(args.warmup)
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        tune = b.autotune(reps=3, cache=os.path.join(td, "tune.txt"))
    chosen = tune["variant"]
    b.step(1)  # captures the step with the chosen launch configurations
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stop = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            start[s].record(stream)
            b.step_async(1)
            stop[s].record(stream)
        b.synchronize()
        torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(z) for a, z in zip(start, stop)), dist)
    value = aggregate_rate(ncell, args.steps, ms, world)
    # per-kernel times: the same number of steps launched kernel by kernel
    b.profile_enable(True)
    b.step(args.steps)
    prof = b.profile_read()
    b.profile_enable(False)
    ngroups = b.num_groups()
    b.close()
    for g in grids:
        g.close()
    sbytes = sum(state_bytes(c, prec) for c in members)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms = kinds[dom][0] / kinds[dom][1]
    algo = 2 * sbytes if dom.startswith("sweep") or dom == "sources" else sbytes
    peak, peak_kind = read_peaks()
    achieved = algo / (dom_ms * 1e-3) / 1e9
    # the same members one at a time: FP32-split, and the plain FP64 path
    k1 = max(1, min(args.steps, 10))
    ms32 = time_alone(members, W.FP32_SPLIT, k1, stream)
    k64 = max(1, min(args.steps, args.fp64_steps, 3))
    ms64 = time_alone(members, W.FP64, k64, stream)
    alone32 = ncell * k1 / (ms32 * 1e-3)
    alone64 = ncell * k64 / (ms64 * 1e-3)
    # end to end through the C ABI: upload every member's initial state,
    # batch, K steps, read every member back
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eg = [mmfrac.Grid(c, prec, stream=stream.cuda_stream) for c in members]
    eb = mmfrac.Batch(eg, stream=stream.cuda_stream)
    eb.step(args.steps)
    outs = [g.read() for g in eg]
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    eb.close()
    for g in eg:
        g.close()
    h2d = sum(c.prim.nbytes + (c.phi0.nbytes if c.phi0 is not None else 0) for c in members)
    d2h = sum(o.nbytes for o in outs)
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == W.FP32_SPLIT else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["ensemble_2d"].format(n=m), "members": m,
                   "cells": ncell, "precision": args.precision,
                   "tile_variants": chosen[:2], "cta_per_sm": tune["cta_per_sm"][:2],
                   "member_groups": ngroups,
                   "l2": "state larger than L2", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "algorithmic_bytes_per_launch": algo,
                     "avg_launch_ms": dom_ms},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kinds.items()},
        "one_at_a_time": {
            "fp32split": {"value": alone32, "ms_per_step": ms32 / k1, "steps": k1},
            "fp64": {"value": alone64, "ms_per_step": ms64 / k64, "steps": k64},
            "batched_over_fp64": value / alone64, "batched_over_fp32split": value / alone32},
        "e2e": {"value": world * ncell * args.steps / e2e_s, "unit": "cell-updates/s",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
        "clocks": clk.summary(),
        "gpu_launches": args.steps * (3 + 2),
    }
    if nested:
        return line
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline("ensemble_2d", m)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_serve(args, rank: int, world: int, nested: bool = False):
    """The served-runs line; nested: returned instead of printed."""
    import torch
    from paper_2210_04037_gb300 import mmfrac
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    count = (args.size if not nested else 0) or DEFAULT_SIZE["serve"]
    reqs = serve_requests(count, seed=7 + rank)
    cases = [serve_case(k, n, 200 + i) for i, (k, n, _, _) in enumerate(reqs)]
    work = [c.ncell * st for c, (_, _, st, _) in zip(cases, reqs)]
    srv = mmfrac.Server(steps_per_tick=8)
    # warm-up: one small run of each dimension (first launches, graph capture)
    for c in (W.spall_1d(1000), W.ring_2d(128), W.cylinder_3d(32)):
        srv.wait(srv.submit(c, 4), timeout=600)
    ids = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for c, (_, _, st, ta) in zip(cases, reqs):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(c, st))
        infos = [srv.wait(rid, timeout=1800)[0] for rid in ids]
    srv.close()
    lat = np.array([i["done_s"] - i["submit_s"] for i in infos])
    span = max(i["done_s"] for i in infos) - min(i["submit_s"] for i in infos)
    value = sum(work) / span
    # one at a time, first come first served: each run's service time alone
    # (create, upload, steps, read back), replayed against the same arrivals
    service = []
    for c, (_, _, st, _) in zip(cases, reqs):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        g = mmfrac.Grid(c, W.FP32_SPLIT)
        g.step_async(st)
        g.read()
        g.close()
        service.append(time.perf_counter() - t1)
    arrive = [i["submit_s"] for i in infos]
    finish, fifo_lat = 0.0, []
    for a, sv in zip(arrive, service):
        finish = max(finish, a) + sv
        fifo_lat.append(finish - a)
    fifo_span = finish - min(arrive)
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": count, "warmup": 3, "ms_per_step": 1e3 * span / count,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["serve"].format(n=count), "requests": count,
                   "mix": {k: sum(1 for r in reqs if r[0] == k) for k in ("1d", "2d", "3d")},
                   "precision": "fp32split", "steps_per_tick": 8,
                   "note": "steps = requests; ms_per_step = makespan per request",
                   "parallelism": f"replicas x{world}"},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "makespan_s": span,
        "one_at_a_time_fifo": {"value": sum(work) / fifo_span, "makespan_s": fifo_span,
                               "p50": float(np.percentile(fifo_lat, 50)),
                               "p99": float(np.percentile(fifo_lat, 99))},
        "roofline": None,
        "clocks": clk.summary(),
    }
    if nested:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_gpu(args, rank: int, world: int):
    import torch
    from paper_2210_04037_gb300 import mmfrac
    if args.workload == "ensemble_2d":
        return run_ensemble(args, rank, world)
    if args.workload == "serve":
        return run_serve(args, rank, world)
    if args.workload == "fragments":
        return run_fragments(args, rank, world)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.size or DEFAULT_SIZE[args.workload]
    case = make_case(args.workload, n)
    prec = W.FP32_SPLIT if args.precision == "fp32split" else W.FP64
    # a dedicated stream: the library orders its work on it and the timing
    # events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sbytes = state_bytes(case, prec)
    flush = None
    if 2 * sbytes < 2 * L2_BYTES:
        flush = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # the timed pass (events around each step only), then the same steps
        # again with events around each launch for the per-kernel times
        xt = 1 if args.x_transport == "weno3rk3" else 0
        g, ms, _, launches = time_device(case, prec, args.steps, args.warmup, stream, flush,
                                         profile=False, x_transport=xt)
        gk, ms_k, prof, _ = time_device(case, prec, args.steps, args.warmup, stream, flush,
                                        profile=True, x_transport=xt)
        gk.close()
        torch.cuda.synchronize()
    ms = max_over_ranks(ms, dist)
    value = aggregate_rate(case.ncell, args.steps, ms, world)
    # dominant kernel and its roofline (algorithmic bytes: one read and one
    # write of the state per launch for the sweeps and the sources)
    peak, peak_kind = read_peaks()
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms = kinds[dom][0] / kinds[dom][1]
    per_pass = algo_bytes_per_pass(case, prec)
    # a sweep and the source step each read and write the state once; the
    # CFL reduction and the totals read it once
    algo = per_pass * case.ncell if dom.startswith("sweep") or dom == "sources" \
        else per_pass * case.ncell // 2
    layout = 2 * sbytes if dom.startswith("sweep") or dom == "sources" else sbytes
    achieved = algo / (dom_ms * 1e-3) / 1e9
    step_bytes = per_pass * case.layout.dim * case.ncell
    step_achieved = step_bytes * args.steps / (ms * 1e-3) / 1e9
    fp32_state = g.read()
    g.close()
    # FP64 beside it (same workload, same steps) and the FP32-split error
    fp64 = None
    if prec == W.FP32_SPLIT and not args.no_fp64:
        k64 = max(1, min(args.steps, args.fp64_steps))
        g64, ms64, prof64, _ = time_device(case, W.FP64, k64, args.warmup, stream, flush,
                                           profile=False)
        fp64 = {"value": world * case.ncell * k64 / (ms64 * 1e-3), "ms_per_step": ms64 / k64,
                "steps": k64}
        g64.close()
        ga = mmfrac.Grid(case, W.FP64, stream=stream.cuda_stream)
        ga.step(args.warmup + args.steps)
        ref = ga.read()
        ga.close()
        num = np.abs(fp32_state - ref).sum(axis=1)
        den = np.abs(ref).sum(axis=1)
        rel = np.where(den > 0, num / np.where(den > 0, den, 1), num)
        names = case.layout.names()
        fp64["fp32split_rel_l1_vs_fp64"] = {names[i]: float(rel[i]) for i in range(len(names))}
    # end-to-end through the C ABI with host buffers: upload the initial
    # state from pinned memory, K steps each returning the conserved totals,
    # read the final primitive fields back
    prim_pinned = torch.from_numpy(np.ascontiguousarray(case.prim)).pin_memory()
    out_pinned = torch.empty(case.prim.shape, dtype=torch.float64).pin_memory()
    h = mmfrac.create_grid(case, prec, stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mmfrac.set_materials(h, case, prim=prim_pinned.numpy())
    for _ in range(args.steps):
        # the step is enqueued; reading its totals back is the one wait per step
        mmfrac.step_async(h, 1, case.cfl)
        mmfrac.conserved_totals(h, len(case.materials))
    mmfrac.synchronize(h)  # a failure latched by any step is raised here
    mmfrac.read_fields(h, True, out=out_pinned.numpy())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    mmfrac.destroy(h)
    e2e_s = max_over_ranks(e2e_s, dist)
    h2d = (case.prim.nbytes + (case.phi0.nbytes if case.phi0 is not None else 0)) / args.steps
    d2h = (len(case.materials) + 4) * 8 + out_pinned.numel() * 8 / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == W.FP32_SPLIT else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload].format(n=n), "cells": case.ncell,
                   "precision": args.precision, "x_transport": args.x_transport,
                   "l2": "flushed between steps (256 MiB write)" if flush is not None
                   else "state larger than L2",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": measured_traffic(args.workload, n, args.precision, dom),
                     "algorithmic_bytes_per_launch": algo,
                     "algorithmic_bytes_per_cell": algo / case.ncell,
                     "layout_bytes_per_launch": layout, "avg_launch_ms": dom_ms},
        "step_roofline": {"bytes_per_update": per_pass * case.layout.dim,
                          "achieved": step_achieved, "peak": peak, "unit": "GB/s",
                          "frac": step_achieved / peak},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kinds.items()},
        "ms_per_step_with_kernel_events": ms_k / args.steps,
        "e2e": {"value": world * case.ncell * args.steps / e2e_s, "unit": "cell-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }
    if fp64:
        line["fp64"] = fp64
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.workload, n)
    if args.workload == "cylinder_3d" and not args.no_extra:
        # the batched ensemble and the served runs, measured in the same run
        # (each rank its own replica of them), so that their numbers are
        # taken beside the headline
        line["ensemble_2d"] = run_ensemble(args, rank, world, nested=True, dist=dist)
        line["serve"] = run_serve(args, rank, world, nested=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mmfrac", choices=["mmfrac", "reference"])
    ap.add_argument("--workload", default="cylinder_3d", choices=list(DEFAULT_SIZE))
    ap.add_argument("--precision", default="fp32split", choices=["fp32split", "fp64"])
    ap.add_argument("--size", type=int, default=0)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="cylinder workload: skip the nested ensemble and served-runs lines")
    ap.add_argument("--x-transport", default="sweep", choices=["sweep", "weno3rk3"],
                    help="transport of the Lagrangian coordinates (default: with the sweeps)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
