"""Oracle evaluation of single cells of a full-size grid: the one-step
result at a cell depends only on the cells within two of it along each axis
(MUSCL-Hancock stencil per split sweep, then local sources), so the oracle
steps a small box around the cell with the global dt and keeps its centre.
Initial data only are sliced here; all arithmetic is the oracle's."""
import copy

import numpy as np

from oracle import OracleGrid


def sub_case(case, lo_idx, shape):
    """The cells lo_idx .. lo_idx + shape - 1 of `case` as a case of its own
    (same materials and lattice, transmissive ends)."""
    d = case.dim
    n = list(case.n)[:d]
    sub = copy.copy(case)
    sl = tuple(slice(lo_idx[k], lo_idx[k] + shape[k]) for k in range(d))[::-1]
    grid = case.prim.reshape([case.prim.shape[0]] + n[::-1])
    sub.prim = np.ascontiguousarray(grid[(slice(None),) + sl].reshape(case.prim.shape[0], -1))
    dx = case.dx
    sub.n = list(shape) + [1] * (3 - d)
    sub.lo = [case.lo[k] + lo_idx[k] * dx[k] for k in range(d)] + list(case.lo[d:])
    sub.hi = [sub.lo[k] + shape[k] * dx[k] for k in range(d)] + list(case.hi[d:])
    sub.bc = [0] * (2 * d)
    return sub


def oracle_cfl_dt(case, cfl=None, slab=16):
    """CFL time step of the full initial state, from slabs along the last axis."""
    d = case.dim
    n = list(case.n)[:d]
    smax = 0.0
    for z0 in range(0, n[-1], slab):
        shape = n[:-1] + [min(slab, n[-1] - z0)]
        if shape[-1] < 2:
            shape[-1] = 2
            z0 = n[-1] - 2
        sub = sub_case(case, [0] * (d - 1) + [z0], shape)
        _, s = OracleGrid(sub).cfl_dt(cfl)
        smax = max(smax, s)
    cfl = case.cfl if cfl is None else cfl
    return cfl * min(case.dx) / smax, smax


def one_step_at(case, cell, dt, margin=3):
    """Primitive fields of `cell` (linear index) after one oracle step of dt."""
    d = case.dim
    n = list(case.n)[:d]
    idx = []
    c = cell
    for k in range(d):
        idx.append(c % n[k])
        c //= n[k]
    lo = [i - margin for i in idx]
    assert all(l >= 0 for l in lo) and all(idx[k] + margin < n[k] for k in range(d))
    shape = [2 * margin + 1] * d
    sub = sub_case(case, lo, shape)
    g = OracleGrid(sub)
    g.step(1, dt=dt)
    w = g.read()
    centre = sum(margin * int(np.prod(shape[:k])) for k in range(d))
    return w[:, centre]


def sample_cells(case, count, seed=0, margin=4):
    """Seeded cells away from the boundary: a third in the solid, a third in
    the diffuse interface, a third in the gas."""
    rng = np.random.default_rng(seed)
    d = case.dim
    n = list(case.n)[:d]
    phi = case.prim[case.layout.o_phi]
    coords = np.unravel_index(np.arange(case.ncell), n[::-1])[::-1]
    ok = np.ones(case.ncell, bool)
    for k in range(d):
        ok &= (coords[k] >= margin) & (coords[k] < n[k] - margin)
    out = []
    for sel in (phi > 0.99, (phi > 0.01) & (phi <= 0.99), phi <= 0.01):
        pool = np.flatnonzero(ok & sel)
        if len(pool):
            out += list(rng.choice(pool, size=min(count // 3, len(pool)), replace=False))
    return sorted(int(c) for c in out)
