"""Seeded synthetic inputs shared by the CUDA solver and the CPU oracle.

This package holds no lattice Boltzmann arithmetic: it produces solid masks
(overlapping-sphere porous media, a bounce-back channel) and seeded initial
fields. Every mask is uint8 with shape (nz, ny, nx), i.e. flat index
x + nx*(y + ny*z), 1 = solid.

The sphere medium follows the paper's randomly placed overlapping spheres
(Section 4.3, "Performance for porous geometries"): centres uniform in the
box, periodic minimum-image distance, spheres added until the porosity
reaches the target. The C implementation in ``geometry.c`` is the one used;
``sphere_pack_numpy`` restates it for small cases so the two can be compared.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geometry.c")
_LIB = os.path.join(_HERE, "libgeometry.so")
_lib = None

# Seed convention for the workloads: base + 1000 * workload index + variant.
SEED_BASE = 20231222


def workload_seed(workload_index: int, variant: int = 0) -> int:
    return SEED_BASE + 1000 * int(workload_index) + int(variant)


def build(force: bool = False) -> str:
    """Compiles geometry.c into libgeometry.so next to it (gcc, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.lbmin_sphere_pack.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        lib.lbmin_sphere_pack.restype = ctypes.c_int
        lib.lbmin_splitmix64_fill.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64]
        lib.lbmin_splitmix64_fill.restype = None
        _lib = lib
    return _lib


@dataclass
class PackInfo:
    porosity: float
    spheres: int


def sphere_pack(nx: int, ny: int, nz: int, radius: float, porosity: float, seed: int,
                max_spheres: int = 1 << 40) -> tuple[np.ndarray, PackInfo]:
    """Overlapping-sphere medium; returns (mask[nz,ny,nx] uint8, PackInfo)."""
    lib = _load()
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    info = np.zeros(2, dtype=np.float64)
    rc = lib.lbmin_sphere_pack(mask.ctypes.data, nx, ny, nz, float(radius), float(porosity),
                               ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(max_spheres),
                               info.ctypes.data)
    if rc != 0:
        raise ValueError("sphere_pack: bad arguments")
    return mask, PackInfo(float(info[0]), int(info[1]))


def splitmix64(seed: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.lbmin_splitmix64_fill(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), out.ctypes.data, count)
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0,1) from the top 53 bits of splitmix64 outputs."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def channel(nx: int, ny: int, nz: int) -> np.ndarray:
    """Bounce-back channel: solid planes z=0 and z=nz-1, fluid between."""
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    mask[0] = 1
    mask[nz - 1] = 1
    return mask


def random_mask(nx: int, ny: int, nz: int, solid_fraction: float, seed: int) -> np.ndarray:
    """Independent per-node solid draws (for edge-case and brute-force tests)."""
    u = uniform01(seed, nx * ny * nz).reshape(nz, ny, nx)
    return (u < solid_fraction).astype(np.uint8)


def random_fields(shape: tuple[int, int, int], seed: int, drho_amp: float, u_amp: float,
                  solid: np.ndarray | None = None) -> tuple[np.ndarray, ...]:
    """Seeded (drho, ux, uy, uz) in float64, uniform in [-amp, amp).

    Solid nodes (if a mask is given) get zeros, the state the solver keeps
    on solid nodes.
    """
    n = int(np.prod(shape))
    u = uniform01(seed, 4 * n).reshape(4, *shape)
    drho = drho_amp * (2.0 * u[0] - 1.0)
    ux = u_amp * (2.0 * u[1] - 1.0)
    uy = u_amp * (2.0 * u[2] - 1.0)
    uz = u_amp * (2.0 * u[3] - 1.0)
    out = [drho, ux, uy, uz]
    if solid is not None:
        for a in out:
            a[solid != 0] = 0.0
    return tuple(np.ascontiguousarray(a) for a in out)


def sphere_pack_numpy(nx: int, ny: int, nz: int, radius: float, porosity: float, seed: int,
                      max_spheres: int = 1 << 40) -> tuple[np.ndarray, PackInfo]:
    """Plain numpy restatement of the C generator, for small grids only."""
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    n = nx * ny * nz
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    stream = splitmix64(seed, 3 * 100000)
    pos = 0
    solid = 0
    placed = 0
    phi = 1.0

    def mi(d, L):
        h = 0.5 * L
        d = np.where(d > h, d - L, d)
        d = np.where(d > h, d - L, d)
        d = np.where(d < -h, d + L, d)
        d = np.where(d < -h, d + L, d)
        return d

    while phi > porosity and placed < max_spheres:
        c = (stream[pos:pos + 3] >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        pos += 3
        cx, cy, cz = c[0] * nx, c[1] * ny, c[2] * nz
        d2 = mi(xx - cx, nx) ** 2 + mi(yy - cy, ny) ** 2 + mi(zz - cz, nz) ** 2
        new = (d2 <= radius * radius) & (mask == 0)
        solid += int(new.sum())
        mask[new] = 1
        placed += 1
        phi = (n - solid) / n
    return mask, PackInfo(float(phi), placed)
