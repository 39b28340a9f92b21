"""z-slab decomposition on CPU ranks (gloo, spawned processes): each rank
steps the oracle on its slab with one halo plane on each side and swaps edge
planes with its neighbours before every step (paper_2312_14742_gb300.slab).
The gathered result must equal the single-domain oracle bit for bit, since a
node's update reads only its neighbours' previous state (Section 2.1.2)."""
import os

import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import slab


def problem(q, case):
    nx, ny, nz = 10, 7, 13
    solid, _ = lbm_inputs.sphere_pack(nx, ny, nz, 2.0, 0.75, 4100 + case)
    st = lbm_inputs.random_fields(solid.shape, 4200 + case, 2e-3, 3e-3, solid)
    g = (1e-5, -2e-6, 3e-6)
    return solid, st, g


def _rank(rank, world, port, q, per_z, case, steps, out_q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        solid, st, g = problem(q, case)
        nz = solid.shape[0]
        z0, z1 = slab.bounds(nz, world, rank)
        nl = z1 - z0
        D = oracle.Domain(q, slab.local_mask(solid, z0, z1, per_z), periodic=(1, 0, 0), g=g)
        local = [slab.local_field(a, z0, z1, per_z) for a in st]
        send_recv, has_lo, has_hi = slab.ring_send_recv(rank, world, per_z)

        def get(k):
            return torch.from_numpy(np.ascontiguousarray(np.stack([local[f][k] for f in range(4)])))

        def put(k, plane):
            for f in range(4):
                local[f][k] = plane[f].numpy()

        for _ in range(steps):
            slab.exchange(get, put, nl, send_recv, has_lo, has_hi)
            local = [np.array(a) for a in D.tau1_step(local)]
        out_q.put((rank, z0, [a[1:nl + 1] for a in local]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", (2, 3))
@pytest.mark.parametrize("per_z", (True, False))
def test_slabs_on_gloo_ranks_equal_one_domain(world, per_z):
    import torch.multiprocessing as mp
    q, case, steps = 19, world + (10 if per_z else 0), 12
    solid, st, g = problem(q, case)
    ref = oracle.Domain(q, solid, periodic=(1, 0, 1 if per_z else 0), g=g).tau1_run(st, steps)
    ctx = mp.get_context("spawn")
    out_q = ctx.Queue()
    port = 29600 + (os.getpid() + 7 * world + (1 if per_z else 0)) % 300
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, per_z, case, steps, out_q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out_q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    full = [np.concatenate([g_[2][f] for g_ in got], axis=0) for f in range(4)]
    for f in range(4):
        assert np.array_equal(full[f], ref[f]), f


def test_bounds_cover_the_box():
    for nz in (1, 7, 13, 256):
        for world in (1, 2, 3, 8):
            if world > nz:
                continue
            spans = [slab.bounds(nz, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1


def test_local_mask_halos():
    solid = np.arange(5 * 2 * 3, dtype=np.uint8).reshape(5, 2, 3) % 2
    m = slab.local_mask(solid, 0, 2, periodic_z=True)
    assert np.array_equal(m[0], solid[4]) and np.array_equal(m[3], solid[2])
    m = slab.local_mask(solid, 0, 2, periodic_z=False)
    assert np.all(m[0] == 1) and np.array_equal(m[1:3], solid[0:2]) and np.array_equal(m[3], solid[2])
    m = slab.local_mask(solid, 3, 5, periodic_z=False)
    assert np.all(m[3] == 1) and np.array_equal(m[0], solid[2])
