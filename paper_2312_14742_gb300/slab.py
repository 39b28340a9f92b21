"""z-slab decomposition of one box over ranks (one GPU each).

Tau1 updates every node from the previous state of its neighbours only
(Section 2.1.2: the nodes of a step are independent), so a box cut into
slabs of z planes needs, per step, one exchange: each slab receives the
plane just below and just above it from the neighbouring slabs (the
previous step's state, all four fields). A slab is a box of its own planes
plus one halo plane on each side; the halo planes are overwritten before
every step, so whatever a step leaves in them is never read. The result is
the same, bit for bit, as stepping the whole box.

The global z axis may be periodic (the slabs form a ring) or not (the halo
plane beyond the first and last slab is solid, which is what a
non-periodic face is to the step kernels).

    bounds(nz, world, rank)          -> (z0, z1) planes of a rank
    local_mask(solid, z0, z1, per_z) -> the slab's mask with its halo planes
    exchange(get, put, nl, send_recv, has_lower, has_upper)
                                      -> one halo exchange
    ring_send_recv(rank, world)      -> send_recv over torch.distributed
    GpuSlab                          -> one rank's slab on its GPU (C ABI)
"""
from __future__ import annotations

import numpy as np

from .lbm import Tau1

RECORD_BYTES = {"f64": 32, "f32": 16, "bf16s": 8}


def bounds(nz: int, world: int, rank: int) -> tuple[int, int]:
    """Planes [z0, z1) of rank: as equal as possible, the first nz % world
    ranks one plane longer."""
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def local_planes(nz: int, z0: int, z1: int, periodic_z: bool) -> list[int | None]:
    """Global plane of each local plane (halo below, own planes, halo above);
    None where a halo lies beyond a non-periodic face."""
    out = []
    for z in range(z0 - 1, z1 + 1):
        if 0 <= z < nz:
            out.append(z)
        elif periodic_z:
            out.append(z % nz)
        else:
            out.append(None)
    return out


def local_mask(solid: np.ndarray, z0: int, z1: int, periodic_z: bool) -> np.ndarray:
    """The slab's mask (nl + 2, ny, nx): halo planes from the neighbours, or
    solid beyond a non-periodic face."""
    nz = solid.shape[0]
    planes = local_planes(nz, z0, z1, periodic_z)
    out = np.ones((len(planes),) + solid.shape[1:], dtype=np.uint8)
    for k, z in enumerate(planes):
        if z is not None:
            out[k] = solid[z]
    return np.ascontiguousarray(out)


def local_field(field: np.ndarray, z0: int, z1: int, periodic_z: bool) -> np.ndarray:
    nz = field.shape[0]
    planes = local_planes(nz, z0, z1, periodic_z)
    out = np.zeros((len(planes),) + field.shape[1:], dtype=field.dtype)
    for k, z in enumerate(planes):
        if z is not None:
            out[k] = field[z]
    return np.ascontiguousarray(out)


def exchange(get, put, nl: int, send_recv, has_lower: bool, has_upper: bool) -> None:
    """One halo exchange of a slab of nl own planes (local planes 1..nl, halos
    0 and nl + 1). get(k) returns local plane k; put(k, plane) overwrites it.
    send_recv(first, last) sends the first own plane to the slab below and the
    last to the slab above, and returns (plane from below, plane from above):
    the last own plane of the slab below and the first of the slab above. A
    slab with no neighbour on a side (non-periodic z) keeps its solid halo."""
    from_below, from_above = send_recv(get(1), get(nl))
    if has_lower:
        put(0, from_below)
    if has_upper:
        put(nl + 1, from_above)


def ring_send_recv(rank: int, world: int, periodic_z: bool):
    """send_recv over torch.distributed for tensors (gloo on the CPU, NCCL on
    GPUs): the ranks form a line in z, closed into a ring when z is
    periodic. A rank that is its own neighbour (one rank, periodic) swaps
    locally."""
    import torch
    import torch.distributed as dist

    below = rank - 1 if rank > 0 else (world - 1 if periodic_z else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic_z else None)

    def send_recv(first, last):
        if world == 1:
            return (last.clone(), first.clone()) if periodic_z else (None, None)
        recv_below = torch.empty_like(last) if below is not None else None
        recv_above = torch.empty_like(first) if above is not None else None
        # Every rank sends its first plane (tag 0) before its last (tag 1);
        # the receives are posted in the order the peer sends them, so that a
        # pair of ranks that are each other's neighbour on both sides (two
        # ranks in a ring) match even where tags are not used (NCCL matches
        # the messages between two ranks in order).
        ops = []
        if below is not None:
            ops.append(dist.P2POp(dist.isend, first.contiguous(), below, tag=0))
        if above is not None:
            ops.append(dist.P2POp(dist.isend, last.contiguous(), above, tag=1))
        if above is not None:
            ops.append(dist.P2POp(dist.irecv, recv_above, above, tag=0))
        if below is not None:
            ops.append(dist.P2POp(dist.irecv, recv_below, below, tag=1))
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        return recv_below, recv_above

    return send_recv, below is not None, above is not None


class GpuSlab:
    """Planes [z0, z1) of a (nx, ny, nz) box as one handle of nz1 - z0 + 2
    planes (the two halos included) on the current CUDA device. Halo
    exchanges copy raw state records of one plane between the handle and a
    device buffer (lbm_tau1_copy_plane); F64, F32 and BF16S storage."""

    def __init__(self, q: int, dims, z0: int, z1: int, storage: str = "f32", periodic=(1, 1, 1),
                 g=(0.0, 0.0, 0.0), stream=None, kernel: str = "auto"):
        import torch
        if storage not in RECORD_BYTES:
            raise ValueError("slab exchange needs F64, F32 or BF16S storage")
        nx, ny, nz = (int(d) for d in dims)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.z0, self.z1, self.nl = int(z0), int(z1), int(z1) - int(z0)
        self.periodic_z = bool(periodic[2])
        self.storage = storage
        # the halo planes are refreshed before every step: the slab itself is
        # non-periodic in z
        self.t = Tau1(q, (nx, ny, self.nl + 2), storage=storage, periodic=(periodic[0], periodic[1], 0), g=g,
                      stream=stream, kernel=kernel)
        nbytes = nx * ny * RECORD_BYTES[storage]
        self.bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]

    def set_geometry(self, solid: np.ndarray) -> None:
        self.t.set_geometry(local_mask(solid, self.z0, self.z1, self.periodic_z))

    def set_fields(self, drho, ux, uy, uz) -> None:
        self.t.set_fields(*[local_field(np.asarray(a, dtype=np.float64), self.z0, self.z1, self.periodic_z)
                            for a in (drho, ux, uy, uz)])

    def get(self, k: int):
        buf = self.bufs[0 if k == 1 else 1]
        self.t.copy_plane(k, buf, False)
        return buf

    def put(self, k: int, plane) -> None:
        self.t.copy_plane(k, plane, True)

    def step(self, n: int = 1) -> None:
        self.t.step(n)

    def fields(self):
        """The slab's own planes, (drho, ux, uy, uz) of shape (nl, ny, nx)."""
        return tuple(a[1:self.nl + 1] for a in self.t.get_fields())

    def close(self) -> None:
        self.t.close()


def run_in_process(slabs: list, nsteps: int) -> None:
    """Steps the slabs of one box held by one process (on one device): before
    every step each slab's halos receive its neighbours' edge planes, as the
    ranks would send them. For tests and for a box split on one GPU."""
    w = len(slabs)
    per = slabs[0].periodic_z
    for _ in range(nsteps):
        firsts = [s.get(1).clone() for s in slabs]
        lasts = [s.get(s.nl).clone() for s in slabs]
        for r, s in enumerate(slabs):
            below = r - 1 if r > 0 else (w - 1 if per else None)
            above = r + 1 if r < w - 1 else (0 if per else None)
            if below is not None:
                s.put(0, lasts[below])
            if above is not None:
                s.put(s.nl + 1, firsts[above])
        for s in slabs:
            s.step(1)
