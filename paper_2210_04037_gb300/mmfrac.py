"""Python binding of the mmfrac C ABI (include/mmfrac.h): argument
marshalling only.  Every step of the method runs in the CUDA library; if the
library cannot be loaded or no GPU is present, calls raise ``MMError``.

The functions carry the C names without the ``mm_`` prefix
(``create_grid``, ``set_materials``, ``step``, ``step_async``,
``synchronize``, ``read_fields``, ``conserved_totals``, ``destroy``,
``last_error``); ``Grid`` bundles them for a ``workloads.Case``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
# MMFRAC_LIB selects another build of the library (e.g. a variant under test)
LIB_PATH = os.environ.get("MMFRAC_LIB") or os.path.join(HERE, "libmmfrac.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA = 0, -1, -2, -3
MM_ENONFINITE, MM_ENOCONV, MM_EDT, MM_ETIMEOUT, MM_ESTATE = -4, -5, -6, -7, -8
STATUS_NAMES = {0: "MM_OK", -1: "MM_EINVAL", -2: "MM_ENOMEM", -3: "MM_ECUDA",
                -4: "MM_ENONFINITE", -5: "MM_ENOCONV", -6: "MM_EDT", -7: "MM_ETIMEOUT",
                -8: "MM_ESTATE"}
FP64, FP32_SPLIT = W.FP64, W.FP32_SPLIT


class MMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc", (ctypes.c_int * 2) * 3),
                ("precision", ctypes.c_int), ("n_materials", ctypes.c_int)]


class Tune(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int * 3), ("cta_per_sm", ctypes.c_int * 3),
                ("from_cache", ctypes.c_int), ("size_class", ctypes.c_int)]


class Material(ctypes.Structure):
    _fields_ = [("eos", ctypes.c_int), ("rho0", ctypes.c_double), ("K0", ctypes.c_double),
                ("G0", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("Gamma0", ctypes.c_double), ("gamma_gas", ctypes.c_double),
                ("plasticity", ctypes.c_int), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("c3", ctypes.c_double), ("n_hard", ctypes.c_double), ("edot0", ctypes.c_double),
                ("damage", ctypes.c_int), ("D_crit", ctypes.c_double), ("eps_t", ctypes.c_double),
                ("eps_c", ctypes.c_double), ("alpha_D", ctypes.c_double),
                ("poisson", ctypes.c_double), ("Ddot0", ctypes.c_double),
                ("shear_model", ctypes.c_int), ("Gp", ctypes.c_double),
                ("Gamma1", ctypes.c_double), ("Gamma2", ctypes.c_double),
                ("gamma_s", ctypes.c_double)]


class Init(ctypes.Structure):
    _fields_ = [("prim", ctypes.POINTER(ctypes.c_double)), ("phi0", ctypes.POINTER(ctypes.c_float)),
                ("phi0_n", ctypes.c_int64 * 3), ("phi0_lo", ctypes.c_double * 3),
                ("phi0_h", ctypes.c_double * 3)]


class RunInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("nfield", ctypes.c_int32),
                ("ncell", ctypes.c_int64), ("steps_done", ctypes.c_int64), ("t", ctypes.c_double),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("used_bytes", ctypes.c_uint64),
                ("pending", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("retired", ctypes.c_int64)]


class Fragment(ctypes.Structure):
    _fields_ = [("label", ctypes.c_int64), ("cells", ctypes.c_int64), ("mass", ctypes.c_double)]


class StepInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt_last", ctypes.c_double), ("smax", ctypes.c_double),
                ("steps_done", ctypes.c_int64), ("bad_cell", ctypes.c_int64)]


EXPORTS = ("mm_create_grid", "mm_set_materials", "mm_set_x_transport",
           "mm_set_lagrangian_seeding", "mm_set_tma_loads", "mm_step",
           "mm_step_async", "mm_synchronize",
           "mm_read_fields",
           "mm_conserved_totals", "mm_num_fields", "mm_num_cells", "mm_destroy",
           "mm_last_error", "mm_kernel_launches", "mm_profile_enable", "mm_profile_read",
           "mm_conserved_totals_noalloc", "mm_batch_create", "mm_batch_set_options",
           "mm_batch_step", "mm_batch_autotune", "mm_batch_autotune_ex", "mm_batch_set_grouping",
           "mm_batch_num_groups", "mm_batch_synchronize",
           "mm_batch_destroy", "mm_batch_profile_enable", "mm_batch_profile_read", "mm_server_create",
           "mm_server_submit", "mm_server_wait", "mm_server_stats", "mm_server_destroy")
KERNEL_KINDS = ("cfl", "dt", "sweep_x", "sweep_y", "sweep_z", "sources", "xtransport",
                "frag_mark", "frag_union", "frag_count", "frag_collect")
X_SWEEP, X_WENO3_RK3 = 0, 1

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libmmfrac.so (built by ``paper_2210_04037_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise MMError(MM_ECUDA, f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.mm_create_grid.argtypes = [P(GridDesc), vp, P(vp)]
        lib.mm_set_materials.argtypes = [vp, P(Material), ctypes.c_int, P(Init)]
        lib.mm_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, P(StepInfo)]
        lib.mm_step_async.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        lib.mm_set_x_transport.argtypes = [vp, ctypes.c_int]
        lib.mm_set_x_transport.restype = ctypes.c_int
        lib.mm_set_lagrangian_seeding.argtypes = [vp, ctypes.c_int]
        lib.mm_set_lagrangian_seeding.restype = ctypes.c_int
        lib.mm_set_tma_loads.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
        lib.mm_set_tma_loads.restype = ctypes.c_int
        lib.mm_fragments.argtypes = [vp, ctypes.c_double, P(ctypes.c_int64), ctypes.c_size_t,
                                     P(Fragment), ctypes.c_size_t, P(ctypes.c_int64)]
        lib.mm_fragments.restype = ctypes.c_int
        lib.mm_batch_create.argtypes = [P(vp), ctypes.c_int, vp, P(vp)]
        lib.mm_batch_set_options.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
        lib.mm_batch_step.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        lib.mm_batch_autotune.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
        lib.mm_batch_autotune_ex.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                             P(Tune)]
        lib.mm_batch_set_grouping.argtypes = [vp, ctypes.c_int64]
        lib.mm_batch_set_grouping.restype = ctypes.c_int
        lib.mm_batch_num_groups.argtypes = [vp]
        lib.mm_batch_num_groups.restype = ctypes.c_int
        lib.mm_batch_synchronize.argtypes = [vp]
        lib.mm_batch_destroy.argtypes = [vp]
        lib.mm_batch_profile_enable.argtypes = [vp, ctypes.c_int]
        lib.mm_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, P(vp)]
        lib.mm_server_submit.argtypes = [vp, P(GridDesc), P(Material), ctypes.c_int, P(Init),
                                         ctypes.c_int, ctypes.c_double, P(ctypes.c_int64)]
        lib.mm_server_wait.argtypes = [vp, ctypes.c_int64, ctypes.c_int, P(RunInfo),
                                       P(ctypes.c_double), ctypes.c_size_t]
        lib.mm_server_stats.argtypes = [vp, P(ServerInfo)]
        lib.mm_server_destroy.argtypes = [vp]
        lib.mm_batch_profile_read.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int64),
                                              ctypes.c_int, ctypes.c_int]
        lib.mm_synchronize.argtypes = [vp, P(StepInfo)]
        lib.mm_read_fields.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_double),
                                       ctypes.c_size_t]
        lib.mm_conserved_totals.argtypes = [vp, P(ctypes.c_double), ctypes.c_size_t]
        lib.mm_num_fields.argtypes = [vp]
        lib.mm_num_cells.argtypes = [vp]
        lib.mm_num_cells.restype = ctypes.c_int64
        lib.mm_destroy.argtypes = [vp]
        lib.mm_last_error.restype = ctypes.c_char_p
        lib.mm_kernel_launches.argtypes = [vp]
        lib.mm_kernel_launches.restype = ctypes.c_int64
        lib.mm_profile_enable.argtypes = [vp, ctypes.c_int]
        lib.mm_profile_enable.restype = ctypes.c_int
        lib.mm_profile_read.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int64), ctypes.c_int,
                                        ctypes.c_int]
        lib.mm_profile_read.restype = ctypes.c_int
        lib.mm_conserved_totals_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                                    ctypes.c_int, P(ctypes.c_double), vp, vp]
        lib.mm_conserved_totals_noalloc.restype = ctypes.c_int
        for fn in ("mm_create_grid", "mm_set_materials", "mm_step", "mm_step_async",
                   "mm_synchronize", "mm_read_fields", "mm_conserved_totals", "mm_destroy",
                   "mm_batch_create", "mm_batch_set_options", "mm_batch_step",
                   "mm_batch_autotune", "mm_batch_autotune_ex", "mm_batch_synchronize",
                   "mm_batch_destroy",
                   "mm_batch_profile_enable", "mm_batch_profile_read", "mm_server_create",
                   "mm_server_submit", "mm_server_wait", "mm_server_stats", "mm_server_destroy"):
            getattr(lib, fn).restype = ctypes.c_int
        _lib = lib
        return lib


def last_error() -> str:
    return load().mm_last_error().decode()


def _check(status: int) -> None:
    if status != MM_OK:
        raise MMError(status, last_error())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def material_struct(m) -> Material:
    s = Material()
    for name, typ in Material._fields_:
        setattr(s, name, int(m[name]) if typ is ctypes.c_int else float(m[name]))
    return s


def _desc(case, precision: int) -> GridDesc:
    d = GridDesc()
    d.dim = case.dim
    for k in range(3):
        d.n[k] = int(case.n[k]) if k < case.dim else 1
        d.lo[k] = float(case.lo[k]) if k < case.dim else 0.0
        d.hi[k] = float(case.hi[k]) if k < case.dim else 1.0
        d.bc[k][0] = int(case.bc[2 * k]) if k < case.dim else 0
        d.bc[k][1] = int(case.bc[2 * k + 1]) if k < case.dim else 0
    d.precision = int(precision)
    d.n_materials = len(case.materials)
    return d


def create_grid(case, precision: int = FP64, stream=None) -> ctypes.c_void_p:
    d = _desc(case, precision)
    h = ctypes.c_void_p()
    _check(load().mm_create_grid(ctypes.byref(d), stream, ctypes.byref(h)))
    return h


def _init(case, prim: np.ndarray | None = None):
    """Materials and initial-state structs of a case, with the arrays they
    point into (kept alive by the caller for the call)."""
    mats = (Material * len(case.materials))(*[material_struct(m) for m in case.materials])
    prim = np.ascontiguousarray(case.prim if prim is None else prim, dtype=np.float64)
    init = Init()
    init.prim = _dptr(prim)
    keep = [prim]
    if case.phi0 is not None:
        phi0 = np.ascontiguousarray(case.phi0, dtype=np.float32)
        keep.append(phi0)
        init.phi0 = phi0.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        for k in range(3):
            init.phi0_n[k] = int(case.pn[k])
            init.phi0_lo[k] = float(case.plo[k])
            init.phi0_h[k] = float(case.ph[k])
    return mats, init, keep


def set_materials(grid, case, prim: np.ndarray | None = None) -> None:
    mats, init, keep = _init(case, prim)
    _check(load().mm_set_materials(grid, mats, len(case.materials), ctypes.byref(init)))


def step(grid, n_steps: int, cfl: float) -> dict:
    info = StepInfo()
    _check(load().mm_step(grid, int(n_steps), float(cfl), ctypes.byref(info)))
    return dict(t=info.t, dt_last=info.dt_last, smax=info.smax, steps=info.steps_done,
                bad_cell=info.bad_cell)


def set_x_transport(grid, scheme: int) -> None:
    """X_SWEEP (X carried by the sweeps) or X_WENO3_RK3 (Sec. 3.2.1)."""
    _check(load().mm_set_x_transport(grid, int(scheme)))


def set_lagrangian_seeding(grid, on: bool) -> None:
    """Seeding of X into void before each step (Sec. 3.2.1), grids with a
    void material: on (default) or off."""
    _check(load().mm_set_lagrangian_seeding(grid, 1 if on else 0))


def set_tma_loads(grid, on=None) -> bool:
    """TMA tile loads in the y and z sweeps of 3D FP32-split grids (two
    materials, no void, n[0] a multiple of 4): on True (default) / False,
    None to leave the switch.  Returns whether the grid's y and z sweeps use
    them (maps present and the switch on)."""
    active = ctypes.c_int(0)
    _check(load().mm_set_tma_loads(grid, -1 if on is None else (1 if on else 0),
                                   ctypes.byref(active)))
    return bool(active.value)


def step_async(grid, n_steps: int, cfl: float) -> None:
    """Enqueue n_steps steps without waiting; in-step failures are reported
    by the next synchronize / step / read_fields."""
    _check(load().mm_step_async(grid, int(n_steps), float(cfl)))


def synchronize(grid) -> dict:
    info = StepInfo()
    _check(load().mm_synchronize(grid, ctypes.byref(info)))
    return dict(t=info.t, dt_last=info.dt_last, smax=info.smax, steps=info.steps_done,
                bad_cell=info.bad_cell)


def read_fields(grid, primitive: bool = True, field_mask: int = (1 << 64) - 1,
                out: np.ndarray | None = None) -> np.ndarray:
    lib = load()
    nf, nc = lib.mm_num_fields(grid), lib.mm_num_cells(grid)
    nsel = sum(1 for f in range(nf) if field_mask >> f & 1)
    if out is None:
        out = np.empty((nsel, nc))
    _check(lib.mm_read_fields(grid, ctypes.c_uint64(field_mask), 1 if primitive else 0, _dptr(out),
                              out.size))
    return out


def conserved_totals(grid, nmat: int) -> np.ndarray:
    out = np.zeros(nmat + 4)
    _check(load().mm_conserved_totals(grid, _dptr(out), out.size))
    return out


def fragments(grid, theta: float = 0.5, labels: bool = True, max_frags: int | None = None):
    """Fragments at void cut-off theta (mm_fragments): per-cell labels
    (int64, -1 outside fragments; None unless asked for) and, in label order,
    each fragment's label, cell count and mass."""
    ncell = int(load().mm_num_cells(grid))
    lab = np.empty(ncell, dtype=np.int64) if labels else None
    cap = ncell if max_frags is None else int(max_frags)
    recs = (Fragment * max(cap, 1))()
    n = ctypes.c_int64()
    P64 = ctypes.POINTER(ctypes.c_int64)
    _check(load().mm_fragments(grid, float(theta),
                               lab.ctypes.data_as(P64) if labels else None,
                               ncell if labels else 0, recs, cap, ctypes.byref(n)))
    k = min(n.value, cap)
    arr = np.frombuffer(recs, dtype=np.dtype([("label", "<i8"), ("cells", "<i8"),
                                              ("mass", "<f8")]), count=k)
    return lab, dict(n=int(n.value), label=arr["label"].copy(), cells=arr["cells"].copy(),
                     mass=arr["mass"].copy())


def destroy(grid) -> None:
    if grid:
        _check(load().mm_destroy(grid))


def kernel_launches(grid) -> int:
    return int(load().mm_kernel_launches(grid))


def profile_enable(grid, enable: bool = True) -> None:
    _check(load().mm_profile_enable(grid, 1 if enable else 0))


def profile_read(grid, reset: bool = True) -> dict:
    n = len(KERNEL_KINDS)
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _check(load().mm_profile_read(grid, _dptr(ms), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  n, 1 if reset else 0))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}


def conserved_totals_noalloc(d_cons: int, dim: int, ncell: int, n_materials: int,
                             n_plastic: int, dx, d_out: int, stream=None) -> None:
    """Totals of a conserved state held in the caller's device memory
    (``d_cons``: device address of [nfield][ncell] FP64 conserved fields),
    written to the caller's device buffer ``d_out`` (N + 4 doubles), with no
    allocation inside the library: for callers that manage all device memory
    themselves and cannot let a library call cudaMalloc.  Asynchronous on
    ``stream``."""
    dxa = (ctypes.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
    _check(load().mm_conserved_totals_noalloc(ctypes.c_void_p(d_cons), int(dim), int(ncell),
                                              int(n_materials), int(n_plastic), dxa,
                                              ctypes.c_void_p(d_out), stream))


class Grid:
    """A grid built from a ``workloads.Case`` on the current CUDA device."""

    def __init__(self, case, precision: int = FP64, stream=None, x_transport: int = X_SWEEP):
        self.case = case
        self.nmat = len(case.materials)
        self.h = create_grid(case, precision, stream)
        try:
            if x_transport != X_SWEEP:
                set_x_transport(self.h, x_transport)
            set_materials(self.h, case)
        except Exception:
            destroy(self.h)
            self.h = None
            raise

    def set_lagrangian_seeding(self, on: bool) -> None:
        set_lagrangian_seeding(self.h, on)

    def set_tma_loads(self, on=None) -> bool:
        return set_tma_loads(self.h, on)

    def step(self, n_steps: int, cfl: float | None = None) -> dict:
        return step(self.h, n_steps, self.case.cfl if cfl is None else cfl)

    def step_async(self, n_steps: int, cfl: float | None = None) -> None:
        step_async(self.h, n_steps, self.case.cfl if cfl is None else cfl)

    def synchronize(self) -> dict:
        return synchronize(self.h)

    def read(self, primitive: bool = True, field_mask: int = (1 << 64) - 1, out=None) -> np.ndarray:
        return read_fields(self.h, primitive, field_mask, out)

    def totals(self) -> np.ndarray:
        return conserved_totals(self.h, self.nmat)

    def launches(self) -> int:
        return kernel_launches(self.h)

    def fragments(self, theta: float = 0.5, labels: bool = True, max_frags: int | None = None):
        return fragments(self.h, theta, labels, max_frags)

    def close(self) -> None:
        if getattr(self, "h", None):
            destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Grids stepped together (``mm_batch_*``): one launch per kernel kind
    over every member, each member with its own dt; the grids are
    referenced, not owned, and must outlive the batch."""

    def __init__(self, grids, stream=None, use_graph: bool = True, cfl: float | None = None):
        lib = load()
        self.grids = list(grids)
        self.cfl = cfl if cfl is not None else self.grids[0].case.cfl
        arr = (ctypes.c_void_p * len(self.grids))(*[g.h for g in self.grids])
        h = ctypes.c_void_p()
        _check(lib.mm_batch_create(arr, len(self.grids), stream, ctypes.byref(h)))
        self.h = h
        if not use_graph:
            self.set_options(use_graph=False)

    def set_options(self, use_graph: bool = True, tile_variant=None) -> None:
        tv = None if tile_variant is None else (ctypes.c_int * 3)(*tile_variant)
        _check(load().mm_batch_set_options(self.h, 1 if use_graph else 0, tv))

    def step_async(self, n_steps: int, cfl: float | None = None) -> None:
        _check(load().mm_batch_step(self.h, int(n_steps), float(self.cfl if cfl is None else cfl)))

    def synchronize(self) -> None:
        _check(load().mm_batch_synchronize(self.h))

    def step(self, n_steps: int, cfl: float | None = None) -> None:
        self.step_async(n_steps, cfl)
        self.synchronize()

    def set_grouping(self, group_bytes: int = -1) -> None:
        """Members stepped in groups of at most group_bytes of state each
        (0: one group; negative: the default, 60 % of L2)."""
        _check(load().mm_batch_set_grouping(self.h, int(group_bytes)))

    def num_groups(self) -> int:
        return int(load().mm_batch_num_groups(self.h))

    def autotune(self, reps: int = 3, cache: str | None = None, force: bool = False):
        """Search the launch configurations (tile shape x persistent CTAs per
        SM per sweep axis); with `cache`, a choice cached for this device and
        size class is taken without timing, and a timed one is saved there.
        Returns the chosen tile shapes (without `cache`) or the whole
        choice as a dict."""
        if cache is None:
            out = (ctypes.c_int * 3)()
            _check(load().mm_batch_autotune(self.h, int(reps), out))
            return list(out)
        t = Tune()
        _check(load().mm_batch_autotune_ex(self.h, int(reps), cache.encode(), 1 if force else 0,
                                           ctypes.byref(t)))
        return dict(variant=list(t.variant), cta_per_sm=list(t.cta_per_sm),
                    from_cache=bool(t.from_cache), size_class=int(t.size_class))

    def profile_enable(self, on: bool = True) -> None:
        _check(load().mm_batch_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, reset: bool = True) -> dict:
        n = len(KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _check(load().mm_batch_profile_read(self.h, ms, cnt, n, 1 if reset else 0))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}

    def close(self) -> None:
        if getattr(self, "h", None):
            load().mm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Served runs with continuous batching (``mm_server_*``): runs are
    admitted while their device memory fits the budget, stepped together
    with the runs already on the GPU, and retired with their primitive
    fields copied to the host."""

    def __init__(self, memory_budget: int = 0, steps_per_tick: int = 8):
        h = ctypes.c_void_p()
        _check(load().mm_server_create(int(memory_budget), int(steps_per_tick), ctypes.byref(h)))
        self.h = h

    def submit(self, case, n_steps: int, precision: int = FP32_SPLIT,
               cfl: float | None = None) -> int:
        d = _desc(case, precision)
        mats, init, keep = _init(case)
        rid = ctypes.c_int64()
        _check(load().mm_server_submit(self.h, ctypes.byref(d), mats, len(case.materials),
                                       ctypes.byref(init), int(n_steps),
                                       float(case.cfl if cfl is None else cfl), ctypes.byref(rid)))
        return int(rid.value)

    def wait(self, rid: int, timeout: float | None = None):
        """(info, primitive fields [nfield][ncell]) of run rid; raises MMError
        (status MM_ETIMEOUT) if it has not finished within timeout seconds."""
        lib = load()
        info = RunInfo()
        ms = -1 if timeout is None else max(0, int(timeout * 1000))
        _check(lib.mm_server_wait(self.h, int(rid), ms, ctypes.byref(info), None, 0))
        out = np.empty((info.nfield, info.ncell))
        _check(lib.mm_server_wait(self.h, int(rid), 0, ctypes.byref(info), _dptr(out), out.size))
        return {k: getattr(info, k) for k, _ in RunInfo._fields_}, out

    def stats(self) -> dict:
        st = ServerInfo()
        _check(load().mm_server_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerInfo._fields_}

    def close(self) -> None:
        if getattr(self, "h", None):
            load().mm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
