"""ctypes front end of the plain FP64 CPU oracle (``mmfrac_oracle.c``).

Test infrastructure only.  It marshals the seeded initial data of
``paper_2210_04037_gb300.workloads`` into the C oracle and reads results
back; all arithmetic of the method is in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mmfrac_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_lock = threading.Lock()
_lib = None


def compile_oracle(src: str, out: str) -> str:
    """gcc, FP64, no FMA contraction, OpenMP loops; `src` must sit beside
    oracle.h (or find it on the include path given by its directory)."""
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-I", HERE, src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle in place (liboracle.so beside the source)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        return LIB
    return compile_oracle(SRC, LIB)


class Material(ctypes.Structure):
    _fields_ = [("eos", ctypes.c_int), ("rho0", ctypes.c_double),
                ("K0", ctypes.c_double), ("G0", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("Gamma0", ctypes.c_double), ("gamma_gas", ctypes.c_double),
                ("plasticity", ctypes.c_int), ("c1", ctypes.c_double),
                ("c2", ctypes.c_double), ("c3", ctypes.c_double),
                ("n_hard", ctypes.c_double), ("edot0", ctypes.c_double),
                ("damage", ctypes.c_int), ("D_crit", ctypes.c_double),
                ("eps_t", ctypes.c_double), ("eps_c", ctypes.c_double),
                ("alpha_D", ctypes.c_double), ("poisson", ctypes.c_double),
                ("Ddot0", ctypes.c_double), ("shear_model", ctypes.c_int),
                ("Gp", ctypes.c_double), ("Gamma1", ctypes.c_double),
                ("Gamma2", ctypes.c_double), ("gamma_s", ctypes.c_double)]


def material_struct(m) -> Material:
    s = Material()
    for name, typ in Material._fields_:
        setattr(s, name, int(m[name]) if typ is ctypes.c_int else float(m[name]))
    return s


def load():
    """The oracle library (built on first use)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        _lib = _bind(ctypes.CDLL(LIB))
        return _lib


def load_from(path: str):
    """Another build of the oracle source (the tests compile copies with a
    planted mistake to show that the pins catch it)."""
    return _bind(ctypes.CDLL(os.path.abspath(path)))


def _bind(lib):
    P = ctypes.POINTER
    d, i, L = ctypes.c_double, ctypes.c_int, ctypes.c_long
    lib.or_create.restype = ctypes.c_void_p
    lib.or_create.argtypes = [i, P(L), P(d), P(d), P(i), i, P(Material), P(d),
                              P(ctypes.c_float), P(L), P(d), P(d), P(i)]
    lib.or_destroy.argtypes = [ctypes.c_void_p]
    lib.or_nfield.argtypes = [ctypes.c_void_p]
    lib.or_ncell.argtypes = [ctypes.c_void_p]
    lib.or_ncell.restype = L
    lib.or_step.argtypes = [ctypes.c_void_p, i, d, d, P(d)]
    lib.or_cfl_dt.argtypes = [ctypes.c_void_p, d, P(d), P(d)]
    lib.or_read.argtypes = [ctypes.c_void_p, i, P(d)]
    lib.or_write_conserved.argtypes = [ctypes.c_void_p, P(d)]
    lib.or_totals.argtypes = [ctypes.c_void_p, P(d)]
    lib.or_set_threads.argtypes = [i]
    lib.or_set_x_scheme.argtypes = [ctypes.c_void_p, i]
    lib.or_seed_x.argtypes = [ctypes.c_void_p]
    lib.or_set_seed_x.argtypes = [ctypes.c_void_p, i]
    lib.or_fragments.restype = L
    lib.or_fragments.argtypes = [ctypes.c_void_p, d, P(L), P(L), P(L), P(d), L]
    lib.or_thermo.argtypes = [P(Material), d, d, d, P(d)]
    lib.or_hencky.argtypes = [P(d), P(d), P(d), P(d)]
    lib.or_lookup.restype = d
    lib.or_lookup.argtypes = [i, P(ctypes.c_float), P(L), P(d), P(d), P(d)]
    lib.or_eps_thresh.restype = d
    lib.or_eps_thresh.argtypes = [d, d, d, d]
    lib.or_Rt.restype = d
    lib.or_Rt.argtypes = [d, d, d, d, d]
    lib.or_damage_rk4.restype = d
    lib.or_damage_rk4.argtypes = [P(Material), d, d, d, d, d, d, d]
    lib.or_plastic_return_cell.argtypes = [P(Material), i, P(d), P(d), P(d), P(d),
                                           d, d, P(d), P(d)]
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleGrid:
    """One oracle grid built from a ``workloads.Case``."""

    def __init__(self, case, threads: int = 0, lib=None):
        lib = load() if lib is None else lib
        self.lib = lib
        self.case = case
        if threads:
            lib.or_set_threads(threads)
        dim = case.dim
        n = (ctypes.c_long * 3)(*[int(case.n[k]) if k < dim else 1 for k in range(3)])
        lo = (ctypes.c_double * 3)(*[float(case.lo[k]) for k in range(3)])
        hi = (ctypes.c_double * 3)(*[float(case.hi[k]) for k in range(3)])
        bc = (ctypes.c_int * 6)(*(list(case.bc) + [0] * (6 - len(case.bc))))
        mats = (Material * len(case.materials))(*[material_struct(m) for m in case.materials])
        self._prim = np.ascontiguousarray(case.prim, dtype=np.float64)
        st = ctypes.c_int(0)
        if case.phi0 is not None:
            phi0 = np.ascontiguousarray(case.phi0, dtype=np.float32)
            pp = phi0.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
            pn = (ctypes.c_long * 3)(*[int(v) for v in case.pn])
            plo = (ctypes.c_double * 3)(*[float(v) for v in case.plo])
            ph = (ctypes.c_double * 3)(*[float(v) for v in case.ph])
        else:
            pp, pn, plo, ph = None, None, None, None
        self.h = lib.or_create(dim, n, lo, hi, bc, len(case.materials), mats,
                               _dp(self._prim), pp, pn, plo, ph, ctypes.byref(st))
        if not self.h:
            raise ValueError("oracle rejected the grid description")
        self.status = st.value
        self.nfield = lib.or_nfield(self.h)
        self.ncell = lib.or_ncell(self.h)
        if self.status != 0:
            raise ValueError(f"oracle: inadmissible initial state ({self.status})")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.or_destroy(self.h)
            self.h = None

    def set_x_scheme(self, scheme: int) -> None:
        """0: X carried by the sweeps; 1: WENO3 + RK3 (Sec. 3.2.1)."""
        if self.lib.or_set_x_scheme(self.h, int(scheme)) != 0:
            raise ValueError("x scheme must be 0 or 1")

    def seed_x(self) -> None:
        """Lagrangian seeding into void once, on the present state (Sec. 3.2.1)."""
        if self.lib.or_seed_x(self.h) != 0:
            raise RuntimeError("oracle seeding failed")

    def set_seed_x(self, on: bool) -> None:
        """Seeding before every step on (default) or off."""
        self.lib.or_set_seed_x(self.h, 1 if on else 0)

    def step(self, nsteps: int, cfl: float | None = None, dt: float = 0.0) -> dict:
        info = np.zeros(6)
        cfl = self.case.cfl if cfl is None else cfl
        rc = self.lib.or_step(self.h, int(nsteps), float(cfl), float(dt), _dp(info))
        out = dict(t=info[0], dt_last=info[1], smax=info[2], steps=int(info[3]),
                   bad_cell=int(info[4]), half_step_bound=int(info[5]), status=rc)
        if rc != 0:
            raise RuntimeError(f"oracle step failed: {out}")
        return out

    def cfl_dt(self, cfl: float | None = None):
        dt, smax = ctypes.c_double(), ctypes.c_double()
        cfl = self.case.cfl if cfl is None else cfl
        rc = self.lib.or_cfl_dt(self.h, float(cfl), ctypes.byref(dt), ctypes.byref(smax))
        if rc != 0:
            raise RuntimeError("oracle cfl failed")
        return dt.value, smax.value

    def read(self, primitive: bool = True) -> np.ndarray:
        out = np.empty((self.nfield, self.ncell))
        self.lib.or_read(self.h, 1 if primitive else 0, _dp(out))
        return out

    def write_conserved(self, U: np.ndarray) -> None:
        U = np.ascontiguousarray(U, dtype=np.float64)
        self.lib.or_write_conserved(self.h, _dp(U))

    def fragments(self, theta: float = 0.5, max_frag: int | None = None):
        """Fragments of the present state at void cut-off theta (Sec. 4.2, 4.3):
        per-cell labels (smallest cell index of the fragment, -1 outside) and,
        in label order, each fragment's label, cell count and solid mass."""
        PL = ctypes.POINTER(ctypes.c_long)
        labels = np.empty(self.ncell, dtype=np.int64)
        cap = self.ncell if max_frag is None else int(max_frag)
        fl = np.empty(max(cap, 1), dtype=np.int64)
        fc = np.empty(max(cap, 1), dtype=np.int64)
        fm = np.empty(max(cap, 1))
        nf = self.lib.or_fragments(self.h, float(theta), labels.ctypes.data_as(PL),
                                   fl.ctypes.data_as(PL), fc.ctypes.data_as(PL), _dp(fm), cap)
        k = min(nf, cap)
        return labels, dict(n=int(nf), label=fl[:k].copy(), cells=fc[:k].copy(),
                            mass=fm[:k].copy())

    def totals(self) -> np.ndarray:
        out = np.zeros(len(self.case.materials) + 4)
        self.lib.or_totals(self.h, _dp(out))
        return out
