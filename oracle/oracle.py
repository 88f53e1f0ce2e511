"""ctypes wrapper of the plain-C FP64 oracle -- test infrastructure only.

Each function mirrors one C entry point of ``tersoff_oracle.c`` (Sec. 2 of the
paper: Eqs. 1-3 and Algorithm 1; velocity Verlet for the MD driver).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        P = ctypes.c_void_p
        L.oracle_energy_forces.argtypes = [i64, P, P, P, ctypes.c_int, P, P, P, P, P, P]
        L.oracle_energy_forces.restype = ctypes.c_int
        L.oracle_neighbors_brute.argtypes = [i64, P, P, dbl, P, P, i64]
        L.oracle_neighbors_brute.restype = i64
        L.oracle_neighbors_cells.argtypes = [i64, P, P, dbl, P, P, i64]
        L.oracle_neighbors_cells.restype = i64
        L.oracle_kinetic.argtypes = [i64, P, P, P]
        L.oracle_kinetic.restype = dbl
        L.oracle_md_run.argtypes = [i64, P, P, P, P, ctypes.c_int, P, P, dbl, i64, P]
        L.oracle_md_run.restype = ctypes.c_int
        L.oracle_accel_unit.argtypes = []
        L.oracle_accel_unit.restype = dbl
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def neighbors(pos, box, rcut, method="auto"):
    """CSR neighbour list (offsets int64[N+1], idx int32[...]), each list ascending.

    method: "brute" (O(N^2) minimum image), "cells" (linked cells, needs >= 3 cells
    per dimension) or "auto" (cells when possible).
    """
    pos = _f64(pos, (-1, 3))
    box = _f64(box, (3,))
    N = pos.shape[0]
    offsets = np.zeros(N + 1, dtype=np.int64)
    cap = max(16, 32 * N)
    while True:
        idx = np.zeros(cap, dtype=np.int32)
        if method in ("cells", "auto"):
            n = lib().oracle_neighbors_cells(N, _p(pos), _p(box), float(rcut), _p(offsets), _p(idx), cap)
            if n == -2 and method == "auto":
                n = lib().oracle_neighbors_brute(N, _p(pos), _p(box), float(rcut), _p(offsets), _p(idx), cap)
        else:
            n = lib().oracle_neighbors_brute(N, _p(pos), _p(box), float(rcut), _p(offsets), _p(idx), cap)
        if n < 0:
            raise ValueError(f"oracle neighbour search failed ({n})")
        if n <= cap:
            return offsets, idx[:n].copy()
        cap = int(n)


def max_cutoff(table):
    t = np.asarray(table).reshape(-1, 14)
    return float(np.max(t[:, 10] + t[:, 11]))


def energy_forces(pos, types, box, table, nlist=None, virial9=False):
    """E (eV), F[N,3] (eV/A) and the virial (6: xx,yy,zz,xy,xz,yz, or the 3x3 matrix).

    The neighbour list defaults to every pair within the table's largest cutoff.
    """
    pos = _f64(pos, (-1, 3))
    types = _i32(types)
    box = _f64(box, (3,))
    table = _f64(table, (-1, 14))
    nt = round(table.shape[0] ** (1.0 / 3.0))
    assert nt ** 3 == table.shape[0]
    if nlist is None:
        nlist = neighbors(pos, box, max_cutoff(table))
    offsets, idx = nlist
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = _i32(idx) if len(idx) else np.zeros(1, dtype=np.int32)
    N = pos.shape[0]
    F = np.zeros((N, 3))
    W = np.zeros(9)
    E = ctypes.c_double(0.0)
    rc = lib().oracle_energy_forces(N, _p(pos), _p(types), _p(box), nt, _p(table), _p(offsets), _p(idx),
                                    ctypes.byref(E), _p(F), _p(W))
    if rc != 0:
        raise ValueError("oracle_energy_forces failed")
    W = W.reshape(3, 3)
    if virial9:
        return E.value, F, W
    return E.value, F, np.array([W[0, 0], W[1, 1], W[2, 2], W[0, 1], W[0, 2], W[1, 2]])


def kinetic(vel, types, masses):
    vel = _f64(vel, (-1, 3))
    return lib().oracle_kinetic(vel.shape[0], _p(vel), _p(_i32(types)), _p(_f64(masses)))


def accel_unit():
    return lib().oracle_accel_unit()


def md_run(pos, vel, types, box, table, masses, dt, nsteps):
    """Velocity-Verlet NVE; returns (pos, vel, trace[nsteps+1, 2] = (PE, KE))."""
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    types = _i32(types)
    table = _f64(table, (-1, 14))
    nt = round(table.shape[0] ** (1.0 / 3.0))
    trace = np.zeros((nsteps + 1, 2))
    rc = lib().oracle_md_run(pos.shape[0], _p(pos), _p(vel), _p(types), _p(_f64(box, (3,))), nt, _p(table),
                             _p(_f64(masses)), float(dt), int(nsteps), _p(trace))
    if rc != 0:
        raise ValueError("oracle_md_run failed")
    return pos, vel, trace
