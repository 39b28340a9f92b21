"""Python binding of liblbm_tau1.so (ctypes; argument marshalling only).

Every function named ``lbm_tau1_*`` here calls the C entry point of the same
name in include/lbm_tau1.h. ``Tau1`` is a thin owner of one handle that
accepts numpy arrays (host) or torch CUDA tensors (device) and raises
``LbmError`` on a non-OK status. All arithmetic runs in the CUDA kernels;
when the library is missing, ``load()`` raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ETIMEOUT, LBM_EBUSY, LBM_ESTATE = range(8)
STATUS_NAMES = ["LBM_OK", "LBM_EINVAL", "LBM_ENOMEM", "LBM_ECUDA", "LBM_EDIVERGED", "LBM_ETIMEOUT", "LBM_EBUSY",
                "LBM_ESTATE"]
LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 = 9, 19, 27
LBM_F64, LBM_F32, LBM_F16S, LBM_BF16S = range(4)
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "bf16s": LBM_BF16S}
LBM_DENSE, LBM_SPARSE, LBM_COMPACT = 0, 1, 2
LAYOUTS = {"dense": LBM_DENSE, "sparse": LBM_SPARSE, "compact": LBM_COMPACT}
# thresholds f* that lbm_tau1_autotune times for the compact layout (the header's list)
COMPACT_THRESHOLDS = (0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.7, 1.01)
LBM_SCHEME_TAU1, LBM_SCHEME_BGK = 0, 1
LBM_KERNEL_AUTO, LBM_KERNEL_SIMPLE, LBM_KERNEL_TILED = 0, 1, 2
KERNELS = {"auto": LBM_KERNEL_AUTO, "simple": LBM_KERNEL_SIMPLE, "tiled": LBM_KERNEL_TILED}


class lbm_tau1_config(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("storage", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_uint8 * 3), ("kernel", ctypes.c_uint8), ("g", ctypes.c_double * 3),
                ("cuda_stream", ctypes.c_void_p)]


class lbm_tau1_stats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("n_fluid", ctypes.c_int64),
                ("nonfinite", ctypes.c_int64), ("mass", ctypes.c_double), ("drho_sum", ctypes.c_double),
                ("mean_ux_superficial", ctypes.c_double), ("mean_u_fluid", ctypes.c_double * 3),
                ("max_abs_u", ctypes.c_double), ("permeability", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"step": self.step, "n_nodes": self.n_nodes, "n_fluid": self.n_fluid, "nonfinite": self.nonfinite,
                "mass": self.mass, "drho_sum": self.drho_sum, "mean_ux_superficial": self.mean_ux_superficial,
                "mean_u_fluid": tuple(self.mean_u_fluid), "max_abs_u": self.max_abs_u,
                "permeability": self.permeability}


class lbm_tau1_compact_info(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("variant", ctypes.c_int32), ("tile", ctypes.c_int32 * 3),
                ("tiled_ok", ctypes.c_int32),
                ("columns", ctypes.c_int64), ("empty_columns", ctypes.c_int64), ("full_columns", ctypes.c_int64),
                ("tiled_columns", ctypes.c_int64),
                ("listed_columns", ctypes.c_int64), ("tiled_nodes", ctypes.c_int64), ("tiled_fluid", ctypes.c_int64),
                ("listed_nodes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["tile"] = tuple(self.tile)
        return d


class lbm_tau1_batch_config(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("storage", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("graph_steps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hbm_budget", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p)]


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64

# name -> (restype, argtypes); every function declared in include/lbm_tau1.h
SIGNATURES = {
    "lbm_tau1_abi_version": (ctypes.c_int32, []),
    "lbm_tau1_create": (_I, [ctypes.POINTER(lbm_tau1_config), ctypes.POINTER(_H)]),
    "lbm_tau1_set_geometry": (_I, [_H, _P, _I]),
    "lbm_tau1_set_fields": (_I, [_H, _P, _P, _P, _P, _I]),
    "lbm_tau1_get_fields": (_I, [_H, _P, _P, _P, _P, _I]),
    "lbm_tau1_step": (_I, [_H, _I64]),
    "lbm_tau1_reduce": (_I, [_H, ctypes.POINTER(lbm_tau1_stats)]),
    "lbm_tau1_synchronize": (_I, [_H]),
    "lbm_tau1_destroy": (_I, [_H]),
    "lbm_tau1_last_error": (ctypes.c_char_p, [_H]),
    "lbm_tau1_launch_count": (_I64, [_H]),
    "lbm_tau1_set_pressure": (_I, [_H, ctypes.c_int32, ctypes.c_double, ctypes.c_double]),
    "lbm_tau1_copy_plane": (_I, [_H, ctypes.c_int32, _P, ctypes.c_int32]),
    "lbm_tau1_selftest_timeout": (_I, [_H]),
    "lbm_tau1_batch_selftest_timeout": (_I, [_H]),
    "lbm_tau1_set_compact_threshold": (_I, [_H, ctypes.c_double]),
    "lbm_tau1_get_compact_info": (_I, [_H, ctypes.POINTER(lbm_tau1_compact_info)]),
    "lbm_tau1_variant_count": (ctypes.c_int32, [_H]),
    "lbm_tau1_set_variant": (_I, [_H, ctypes.c_int32]),
    "lbm_tau1_autotune": (_I, [_H, ctypes.c_int32, _P, _P]),
    "lbm_tau1_set_tune_cache": (None, [ctypes.c_char_p]),
    "lbm_tau1_batch_create": (_I, [ctypes.POINTER(lbm_tau1_batch_config), ctypes.POINTER(_H)]),
    "lbm_tau1_batch_footprint": (ctypes.c_uint64, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "lbm_tau1_batch_admit": (_I, [_H, ctypes.POINTER(lbm_tau1_config), _P, _I, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_tau1_batch_step": (_I, [_H, _I64]),
    "lbm_tau1_batch_stats": (_I, [_H, ctypes.c_int32, _P, _P]),
    "lbm_tau1_batch_stats_queue": (_I, [_H, ctypes.c_int32, _P]),
    "lbm_tau1_batch_stats_wait": (_I, [_H, _P]),
    "lbm_tau1_batch_get_fields": (_I, [_H, ctypes.c_int32, _P, _P, _P, _P, _I]),
    "lbm_tau1_batch_release": (_I, [_H, ctypes.c_int32]),
    "lbm_tau1_batch_synchronize": (_I, [_H]),
    "lbm_tau1_batch_destroy": (_I, [_H]),
    "lbm_tau1_batch_live": (ctypes.c_int32, [_H]),
    "lbm_tau1_batch_bytes_free": (ctypes.c_uint64, [_H]),
    "lbm_tau1_batch_launch_count": (_I64, [_H]),
    "lbm_tau1_batch_last_error": (ctypes.c_char_p, [_H]),
    "lbm_tau1_reduce_noalloc": (_I, [ctypes.c_int32, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "lbm_tau1_noalloc_last_error": (ctypes.c_char_p, []),
}

_lib = None


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


def load(build_if_missing: bool = False):
    """Loads liblbm_tau1.so. Raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run paper_2312_14742_gb300.build")
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _fn(name):
    return getattr(load(), name)


# ---- the C entry points, same names -------------------------------------------------------

def lbm_tau1_abi_version() -> int:
    return _fn("lbm_tau1_abi_version")()


def lbm_tau1_create(cfg: lbm_tau1_config) -> tuple[int, int | None]:
    h = _H()
    st = _fn("lbm_tau1_create")(ctypes.byref(cfg), ctypes.byref(h))
    return st, h.value


def lbm_tau1_set_geometry(h, solid_ptr, on_device: int) -> int:
    return _fn("lbm_tau1_set_geometry")(h, solid_ptr, on_device)


def lbm_tau1_set_fields(h, drho, ux, uy, uz, on_device: int) -> int:
    return _fn("lbm_tau1_set_fields")(h, drho, ux, uy, uz, on_device)


def lbm_tau1_get_fields(h, drho, ux, uy, uz, on_device: int) -> int:
    return _fn("lbm_tau1_get_fields")(h, drho, ux, uy, uz, on_device)


def lbm_tau1_step(h, nsteps: int) -> int:
    return _fn("lbm_tau1_step")(h, nsteps)


def lbm_tau1_reduce(h, stats: lbm_tau1_stats) -> int:
    return _fn("lbm_tau1_reduce")(h, ctypes.byref(stats))


def lbm_tau1_synchronize(h) -> int:
    return _fn("lbm_tau1_synchronize")(h)


def lbm_tau1_destroy(h) -> int:
    return _fn("lbm_tau1_destroy")(h)


def lbm_tau1_last_error(h) -> str:
    s = _fn("lbm_tau1_last_error")(h)
    return s.decode() if s else ""


def lbm_tau1_launch_count(h) -> int:
    return _fn("lbm_tau1_launch_count")(h)


def lbm_tau1_set_pressure(h, axis: int, rho_lo: float, rho_hi: float) -> int:
    return _fn("lbm_tau1_set_pressure")(h, axis, rho_lo, rho_hi)


def lbm_tau1_copy_plane(h, z: int, buf, to_handle: int) -> int:
    return _fn("lbm_tau1_copy_plane")(h, z, buf, to_handle)


def lbm_tau1_selftest_timeout(h) -> int:
    return _fn("lbm_tau1_selftest_timeout")(h)


def lbm_tau1_batch_selftest_timeout(b) -> int:
    return _fn("lbm_tau1_batch_selftest_timeout")(b)


def lbm_tau1_set_compact_threshold(h, f: float) -> int:
    return _fn("lbm_tau1_set_compact_threshold")(h, f)


def lbm_tau1_get_compact_info(h, out: lbm_tau1_compact_info) -> int:
    return _fn("lbm_tau1_get_compact_info")(h, ctypes.byref(out))


def lbm_tau1_variant_count(h) -> int:
    return _fn("lbm_tau1_variant_count")(h)


def lbm_tau1_set_variant(h, variant: int) -> int:
    return _fn("lbm_tau1_set_variant")(h, variant)


def lbm_tau1_autotune(h, trials: int, chosen=None, ms_per_step=None) -> int:
    return _fn("lbm_tau1_autotune")(h, trials, chosen, ms_per_step)


def lbm_tau1_set_tune_cache(path) -> None:
    _fn("lbm_tau1_set_tune_cache")(None if path is None else os.fsencode(path))


def lbm_tau1_reduce_noalloc(storage, n, drho, ux, uy, uz, inv_scale, solid, g, out, stream) -> int:
    return _fn("lbm_tau1_reduce_noalloc")(storage, n, drho, ux, uy, uz, inv_scale, solid, g, out, stream)


def lbm_tau1_noalloc_last_error() -> str:
    s = _fn("lbm_tau1_noalloc_last_error")()
    return s.decode() if s else ""


def lbm_tau1_batch_create(cfg: lbm_tau1_batch_config) -> tuple[int, int | None]:
    h = _H()
    st = _fn("lbm_tau1_batch_create")(ctypes.byref(cfg), ctypes.byref(h))
    return st, h.value


def lbm_tau1_batch_footprint(storage: int, nx: int, ny: int, nz: int) -> int:
    return _fn("lbm_tau1_batch_footprint")(storage, nx, ny, nz)


def lbm_tau1_batch_admit(b, cfg: lbm_tau1_config, solid_ptr, on_device: int) -> tuple[int, int]:
    slot = ctypes.c_int32(-1)
    st = _fn("lbm_tau1_batch_admit")(b, ctypes.byref(cfg), solid_ptr, on_device, ctypes.byref(slot))
    return st, slot.value


def lbm_tau1_batch_step(b, nsteps: int) -> int:
    return _fn("lbm_tau1_batch_step")(b, nsteps)


def lbm_tau1_batch_stats(b, n: int, slots_ptr, stats_ptr) -> int:
    return _fn("lbm_tau1_batch_stats")(b, n, slots_ptr, stats_ptr)


def lbm_tau1_batch_stats_queue(b, n: int, slots_ptr) -> int:
    return _fn("lbm_tau1_batch_stats_queue")(b, n, slots_ptr)


def lbm_tau1_batch_stats_wait(b, stats_ptr) -> int:
    return _fn("lbm_tau1_batch_stats_wait")(b, stats_ptr)


def lbm_tau1_batch_get_fields(b, slot: int, drho, ux, uy, uz, on_device: int) -> int:
    return _fn("lbm_tau1_batch_get_fields")(b, slot, drho, ux, uy, uz, on_device)


def lbm_tau1_batch_release(b, slot: int) -> int:
    return _fn("lbm_tau1_batch_release")(b, slot)


def lbm_tau1_batch_synchronize(b) -> int:
    return _fn("lbm_tau1_batch_synchronize")(b)


def lbm_tau1_batch_destroy(b) -> int:
    return _fn("lbm_tau1_batch_destroy")(b)


def lbm_tau1_batch_live(b) -> int:
    return _fn("lbm_tau1_batch_live")(b)


def lbm_tau1_batch_bytes_free(b) -> int:
    return _fn("lbm_tau1_batch_bytes_free")(b)


def lbm_tau1_batch_launch_count(b) -> int:
    return _fn("lbm_tau1_batch_launch_count")(b)


def lbm_tau1_batch_last_error(b) -> str:
    s = _fn("lbm_tau1_batch_last_error")(b)
    return s.decode() if s else ""


# ---- convenience owner of one handle ---------------------------------------------------------

def _ptr(a, on_device: bool):
    if a is None:
        return None
    if on_device:
        return a.data_ptr()
    return a.ctypes.data


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


class Tau1:
    """One box: ``Tau1(q, (nx, ny, nz), storage="f32", periodic=(1,1,1), g=(gx,0,0))``."""

    def __init__(self, q: int, dims, storage: str = "f32", periodic=(1, 1, 1), g=(0.0, 0.0, 0.0),
                 kernel: str = "auto", stream=None, scheme: int = LBM_SCHEME_TAU1, layout=LBM_DENSE):
        nx, ny, nz = (int(d) for d in dims)
        if isinstance(layout, str):
            layout = LAYOUTS[layout]
        cfg = lbm_tau1_config()
        cfg.q, cfg.storage, cfg.layout, cfg.scheme = int(q), STORAGE[storage], int(layout), int(scheme)
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        for a in range(3):
            cfg.periodic[a] = 1 if periodic[a] else 0
            cfg.g[a] = float(g[a])
        cfg.kernel = KERNELS[kernel]
        cfg.cuda_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        st, h = lbm_tau1_create(cfg)
        if st != LBM_OK:
            raise LbmError(st, lbm_tau1_last_error(None))
        self.h = h
        self.dims = (nx, ny, nz)
        self.shape = (nz, ny, nx)
        self.q = int(q)
        self.storage = storage
        self.g = tuple(float(x) for x in g)

    def _check(self, st: int) -> int:
        if st != LBM_OK:
            raise LbmError(st, lbm_tau1_last_error(self.h))
        return st

    def set_geometry(self, solid) -> None:
        dev = _is_device(solid)
        if not dev:
            solid = np.ascontiguousarray(solid, dtype=np.uint8)
        assert solid.numel() if dev else solid.size == self.dims[0] * self.dims[1] * self.dims[2]
        self._keep = solid
        self._check(lbm_tau1_set_geometry(self.h, _ptr(solid, dev), 1 if dev else 0))

    def set_fields(self, drho, ux, uy, uz) -> None:
        arrs = [drho, ux, uy, uz]
        dev = _is_device(drho)
        if not dev:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        self._check(lbm_tau1_set_fields(self.h, *[_ptr(a, dev) for a in arrs], 1 if dev else 0))

    def get_fields(self, out=None):
        """Returns (drho, ux, uy, uz) as float64 numpy arrays (nz, ny, nx), or fills the
        given torch CUDA tensors."""
        if out is not None:
            self._check(lbm_tau1_get_fields(self.h, *[_ptr(a, True) for a in out], 1))
            return out
        arrs = [np.empty(self.shape, dtype=np.float64) for _ in range(4)]
        self._check(lbm_tau1_get_fields(self.h, *[_ptr(a, False) for a in arrs], 0))
        return tuple(arrs)

    def step(self, nsteps: int = 1) -> None:
        self._check(lbm_tau1_step(self.h, int(nsteps)))

    def copy_plane(self, z: int, buf, to_handle: bool) -> None:
        """Raw records of plane z of the current state to (to_handle False) or
        from (True) a device buffer (a torch CUDA tensor of nx*ny*record bytes)."""
        self._check(lbm_tau1_copy_plane(self.h, int(z), _ptr(buf, True), 1 if to_handle else 0))

    def set_pressure(self, axis: int, rho_lo: float, rho_hi: float) -> None:
        """Constant-density (Zou-He) faces on a non-periodic axis (-1: none)."""
        self._check(lbm_tau1_set_pressure(self.h, int(axis), float(rho_lo), float(rho_hi)))

    def set_compact_threshold(self, f: float) -> None:
        """Compact layout: fluid fraction f* from which a tile column goes to
        the tiled kernel (the lists are rebuilt; the state is unchanged)."""
        self._check(lbm_tau1_set_compact_threshold(self.h, float(f)))

    def compact_info(self) -> dict:
        """Compact layout: how the box is split (tile columns per class, nodes)."""
        s = lbm_tau1_compact_info()
        self._check(lbm_tau1_get_compact_info(self.h, s))
        return s.as_dict()

    def reduce(self, allow_diverged: bool = False) -> dict:
        s = lbm_tau1_stats()
        st = lbm_tau1_reduce(self.h, s)
        if st == LBM_EDIVERGED and allow_diverged:
            d = s.as_dict()
            d["diverged"] = True
            return d
        self._check(st)
        return s.as_dict()

    def synchronize(self) -> None:
        self._check(lbm_tau1_synchronize(self.h))

    def autotune(self, trials: int = 20) -> tuple[int, float]:
        """Times each tile-shape variant (compact layout: each threshold of
        COMPACT_THRESHOLDS); keeps the fastest. Returns (index, ms per step)."""
        ch = ctypes.c_int32(0)
        ms = ctypes.c_float(0)
        self._check(lbm_tau1_autotune(self.h, int(trials), ctypes.byref(ch), ctypes.byref(ms)))
        return ch.value, ms.value

    def set_variant(self, v: int) -> None:
        self._check(lbm_tau1_set_variant(self.h, int(v)))

    @property
    def variant_count(self) -> int:
        return lbm_tau1_variant_count(self.h)

    @property
    def launch_count(self) -> int:
        return lbm_tau1_launch_count(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            lbm_tau1_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def box_config(q: int, dims, storage: str, periodic=(1, 1, 1), g=(0.0, 0.0, 0.0)) -> lbm_tau1_config:
    """lbm_tau1_config of one dense Tau1 box."""
    cfg = lbm_tau1_config()
    cfg.q, cfg.storage, cfg.layout, cfg.scheme = int(q), STORAGE[storage], LBM_DENSE, LBM_SCHEME_TAU1
    cfg.nx, cfg.ny, cfg.nz = (int(d) for d in dims)
    for a in range(3):
        cfg.periodic[a] = 1 if periodic[a] else 0
        cfg.g[a] = float(g[a])
    return cfg


class Batch:
    """Boxes stepped together: ``Batch(19, "f32", capacity=64)``; ``admit`` returns a slot
    (or None when the box does not fit now), ``step(n)`` advances every live box."""

    def __init__(self, q: int, storage: str = "f32", capacity: int = 64, variant: int = 0, graph_steps: int = 100,
                 hbm_budget: int = 0, stream=None):
        cfg = lbm_tau1_batch_config()
        cfg.q, cfg.storage, cfg.variant, cfg.capacity = int(q), STORAGE[storage], int(variant), int(capacity)
        cfg.graph_steps, cfg.hbm_budget = int(graph_steps), int(hbm_budget)
        cfg.cuda_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        st, b = lbm_tau1_batch_create(cfg)
        if st != LBM_OK:
            raise LbmError(st, lbm_tau1_last_error(None))
        self.b = b
        self.q = int(q)
        self.storage = storage
        self.shapes: dict[int, tuple] = {}

    def _check(self, st: int) -> int:
        if st != LBM_OK:
            raise LbmError(st, lbm_tau1_batch_last_error(self.b))
        return st

    @staticmethod
    def footprint(storage: str, dims) -> int:
        return lbm_tau1_batch_footprint(STORAGE[storage], *(int(d) for d in dims))

    def admit(self, solid, periodic=(1, 1, 1), g=(0.0, 0.0, 0.0)):
        """solid: uint8 array (nz, ny, nx), host or torch CUDA. Returns the slot, or None
        if the batch is full or the footprint does not fit (LBM_EBUSY)."""
        dev = _is_device(solid)
        if not dev:
            solid = np.ascontiguousarray(solid, dtype=np.uint8)
        nz, ny, nx = solid.shape
        cfg = box_config(self.q, (nx, ny, nz), self.storage, periodic, g)
        st, slot = lbm_tau1_batch_admit(self.b, cfg, _ptr(solid, dev), 1 if dev else 0)
        if st == LBM_EBUSY:
            return None
        self._check(st)
        self.shapes[slot] = (nz, ny, nx)
        return slot

    def step(self, nsteps: int = 1) -> None:
        self._check(lbm_tau1_batch_step(self.b, int(nsteps)))

    def stats(self, slots, allow_diverged: bool = False) -> list[dict]:
        slots = list(slots)
        n = len(slots)
        if n == 0:
            return []
        arr = (ctypes.c_int32 * n)(*slots)
        out = (lbm_tau1_stats * n)()
        st = lbm_tau1_batch_stats(self.b, n, ctypes.cast(arr, _P), ctypes.cast(out, _P))
        if not (st == LBM_EDIVERGED and allow_diverged):
            self._check(st)
        return [o.as_dict() for o in out]

    def stats_queue(self, slots) -> None:
        """Queues the statistics of the given live slots and returns without
        waiting; stats_wait() takes them (steps, releases and admissions may
        be queued in between)."""
        slots = list(slots)
        arr = (ctypes.c_int32 * max(1, len(slots)))(*slots)
        self._check(lbm_tau1_batch_stats_queue(self.b, len(slots), ctypes.cast(arr, _P)))
        self._queued = len(slots)

    def stats_wait(self, allow_diverged: bool = False) -> list[dict]:
        """The statistics queued by stats_queue, in the order of its slots."""
        n = getattr(self, "_queued", 0)
        out = (lbm_tau1_stats * max(1, n))()
        st = lbm_tau1_batch_stats_wait(self.b, ctypes.cast(out, _P))
        self._queued = 0
        if not (st == LBM_EDIVERGED and allow_diverged):
            self._check(st)
        return [out[i].as_dict() for i in range(n)]

    def get_fields(self, slot: int):
        arrs = [np.empty(self.shapes[slot], dtype=np.float64) for _ in range(4)]
        self._check(lbm_tau1_batch_get_fields(self.b, int(slot), *[_ptr(a, False) for a in arrs], 0))
        return tuple(arrs)

    def release(self, slot: int) -> None:
        self._check(lbm_tau1_batch_release(self.b, int(slot)))
        self.shapes.pop(slot, None)

    def synchronize(self) -> None:
        self._check(lbm_tau1_batch_synchronize(self.b))

    @property
    def live(self) -> int:
        return lbm_tau1_batch_live(self.b)

    @property
    def bytes_free(self) -> int:
        return lbm_tau1_batch_bytes_free(self.b)

    @property
    def launch_count(self) -> int:
        return lbm_tau1_batch_launch_count(self.b)

    def close(self) -> None:
        if getattr(self, "b", None):
            lbm_tau1_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
