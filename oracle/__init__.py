"""FP64 CPU oracle for Tau1 and standard BGK (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg use this package. The CUDA path never imports it.

The arithmetic lives in ``tau1_oracle.c`` (plain C, FP64, no FMA
contraction); this module only marshals numpy arrays into it. Arrays use the
layout (nz, ny, nx), i.e. flat index x + nx*(y + ny*z). State is
(drho, ux, uy, uz) with drho = rho - 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tau1_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NU = 1.0 / 6.0  # kinematic viscosity at tau = 1: c_s^2 (tau - 1/2)


def build(force: bool = False, src: str = _SRC, out: str = _LIB, openmp: bool = True) -> str:
    """Compiles the oracle with gcc. Returns the shared-library path."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
        if openmp:
            cmd.append("-fopenmp")
        cmd += [src, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_I64 = ctypes.c_int64


def load(path: str | None = None):
    """Loads (building if needed) the oracle library and declares signatures."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    lib = ctypes.CDLL(path or build())
    lib.orc_lattice.argtypes = [_I, _P, _P, _P]
    lib.orc_feq_dev.argtypes = [_I, _I, _D, _D, _D, _D]
    lib.orc_feq_dev.restype = _D
    lib.orc_tau1_step.argtypes = [_I, _I, _I, _I, _P, _P, _P] + [_P] * 8
    lib.orc_tau1_run.argtypes = [_I, _I, _I, _I, _P, _P, _P] + [_P] * 4 + [_I64]
    lib.orc_tau1_step_bc.argtypes = [_I, _I, _I, _I, _P, _P, _P, _P] + [_P] * 8
    lib.orc_tau1_run_bc.argtypes = [_I, _I, _I, _I, _P, _P, _P, _P] + [_P] * 4 + [_I64]
    lib.orc_tau1_nodes.argtypes = [_I, _I, _I, _I, _P, _P, _P] + [_P] * 4 + [_P, _I64, _P]
    lib.orc_bgk_init.argtypes = [_I, _I, _I, _I, _P, _D, _P] + [_P] * 4 + [_P]
    lib.orc_bgk_step.argtypes = [_I, _I, _I, _I, _P, _P, _D, _P, _P, _P] + [_P] * 4
    lib.orc_reduce.argtypes = [_I, _I, _I, _P, _P] + [_P] * 4 + [_P]
    lib.orc_set_threads.argtypes = [_I]
    lib.orc_set_threads.restype = None
    lib.orc_get_threads.restype = _I
    if path is None:
        _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Domain:
    """Geometry and driving of one box: lattice q (9 = D2Q9, one plane), mask
    (nz,ny,nx), periodicity, g, and optional constant-density (Zou-He)
    faces ``pressure = (axis, rho at coordinate 0, rho at coordinate n-1)``
    on a non-periodic axis."""

    def __init__(self, q: int, solid: np.ndarray, periodic=(1, 1, 1), g=(0.0, 0.0, 0.0), lib=None, pressure=None):
        self.q = int(q)
        self.solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.nz, self.ny, self.nx = self.solid.shape
        self.periodic = np.asarray(periodic, dtype=np.int32)
        self.g = np.asarray(g, dtype=np.float64)
        self.bc = np.asarray(pressure if pressure is not None else (-1.0, 1.0, 1.0), dtype=np.float64)
        self.lib = lib or load()

    @property
    def shape(self):
        return self.solid.shape

    def _args(self):
        return (self.q, self.nx, self.ny, self.nz, self.periodic.ctypes.data, self.g.ctypes.data,
                self.solid.ctypes.data)

    def _args_bc(self):
        return (self.q, self.nx, self.ny, self.nz, self.periodic.ctypes.data, self.g.ctypes.data,
                self.bc.ctypes.data, self.solid.ctypes.data)

    def zero_state(self):
        z = np.zeros(self.shape, dtype=np.float64)
        return (z, z.copy(), z.copy(), z.copy())

    def tau1_step(self, state):
        s = [_f64(a) for a in state]
        o = [np.empty(self.shape, dtype=np.float64) for _ in range(4)]
        rc = self.lib.orc_tau1_step_bc(*self._args_bc(), *[a.ctypes.data for a in s], *[a.ctypes.data for a in o])
        if rc != 0:
            raise ValueError("orc_tau1_step failed")
        return tuple(o)

    def tau1_run(self, state, nsteps: int):
        s = [np.array(a, dtype=np.float64, order="C", copy=True) for a in state]
        rc = self.lib.orc_tau1_run_bc(*self._args_bc(), *[a.ctypes.data for a in s], int(nsteps))
        if rc != 0:
            raise ValueError("orc_tau1_run failed")
        return tuple(s)

    def tau1_nodes(self, state, nodes):
        """One step evaluated at the flat node indices; returns [count,4]."""
        s = [_f64(a) for a in state]
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        out = np.empty((len(nodes), 4), dtype=np.float64)
        rc = self.lib.orc_tau1_nodes(*self._args(), *[a.ctypes.data for a in s], nodes.ctypes.data,
                                     len(nodes), out.ctypes.data)
        if rc != 0:
            raise ValueError("orc_tau1_nodes failed")
        return out

    def bgk_init(self, state, tau: float = 1.0):
        s = [_f64(a) for a in state]
        h = np.empty((self.q,) + self.shape, dtype=np.float64)
        rc = self.lib.orc_bgk_init(self.q, self.nx, self.ny, self.nz, self.g.ctypes.data, float(tau),
                                   self.solid.ctypes.data, *[a.ctypes.data for a in s], h.ctypes.data)
        if rc != 0:
            raise ValueError("orc_bgk_init failed")
        return h

    def bgk_step(self, h, tau: float = 1.0):
        h = _f64(h)
        ho = np.empty_like(h)
        o = [np.empty(self.shape, dtype=np.float64) for _ in range(4)]
        rc = self.lib.orc_bgk_step(*self._args()[:6], float(tau), self.solid.ctypes.data, h.ctypes.data,
                                   ho.ctypes.data, *[a.ctypes.data for a in o])
        if rc != 0:
            raise ValueError("orc_bgk_step failed")
        return ho, tuple(o)

    def reduce(self, state) -> dict:
        s = [_f64(a) for a in state]
        out = np.empty(9, dtype=np.float64)
        self.lib.orc_reduce(self.nx, self.ny, self.nz, self.g.ctypes.data, self.solid.ctypes.data,
                            *[a.ctypes.data for a in s], out.ctypes.data)
        return {"n_fluid": int(out[0]), "mass": out[1], "mean_ux_superficial": out[2],
                "mean_u_fluid": tuple(out[3:6]), "max_abs_u": out[6], "permeability": out[7],
                "nonfinite": int(out[8])}


def lattice(q: int, lib=None):
    """(c[q,3] int, w[q] float64, inv[q] int) as the oracle types them."""
    lib = lib or load()
    c = np.empty((q, 3), dtype=np.int32)
    w = np.empty(q, dtype=np.float64)
    inv = np.empty(q, dtype=np.int32)
    if lib.orc_lattice(q, c.ctypes.data, w.ctypes.data, inv.ctypes.data) != 0:
        raise ValueError(f"no lattice with q = {q}")
    return c, w, inv


def feq_dev(q: int, k: int, drho: float, vx: float, vy: float, vz: float, lib=None) -> float:
    lib = lib or load()
    return lib.orc_feq_dev(q, k, drho, vx, vy, vz)


def set_threads(n: int) -> None:
    load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(load().orc_get_threads())
