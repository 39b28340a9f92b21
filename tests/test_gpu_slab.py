"""z-slabs of one box on one GPU, stepped in one process with the halo
exchange of the decomposition (lbm_tau1_copy_plane between the slabs'
handles): the same bits as the whole box on the same GPU."""
import numpy as np
import pytest

import lbm_inputs
from paper_2312_14742_gb300 import Tau1, build, slab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.mark.parametrize("storage", ("f64", "f32", "bf16s"))
@pytest.mark.parametrize("world,per_z", [(2, True), (3, False), (4, True)])
def test_slabs_equal_one_domain(storage, world, per_z):
    """FP64 and FP32: the same bits. BF16 stores round stochastically with
    bits hashed from the node's index in its handle, which differs between a
    slab and the whole box, so the two runs agree to that rounding noise:
    every velocity within 3 % of the largest, the mean difference within
    0.1 %."""
    nx, ny, nz = 64, 24, 37
    solid, _ = lbm_inputs.sphere_pack(nx, ny, nz, 3.0, 0.8, 4300 + world)
    st = lbm_inputs.random_fields(solid.shape, 4301, 2e-3, 3e-3, solid)
    g = (1e-5, 0.0, -2e-6)
    per = (1, 1, 1 if per_z else 0)
    with Tau1(19, (nx, ny, nz), storage=storage, periodic=per, g=g) as t:
        t.set_geometry(solid)
        t.set_fields(*st)
        t.step(20)
        ref = t.get_fields()
    slabs = [slab.GpuSlab(19, (nx, ny, nz), *slab.bounds(nz, world, r), storage=storage, periodic=per, g=g)
             for r in range(world)]
    try:
        for s in slabs:
            s.set_geometry(solid)
            s.set_fields(*st)
        slab.run_in_process(slabs, 20)
        got = [np.concatenate([s.fields()[f] for s in slabs], axis=0) for f in range(4)]
    finally:
        for s in slabs:
            s.close()
    for f in range(4):
        if storage == "bf16s":
            scale = float(np.max(np.abs(ref[f]))) or 1.0
            assert np.max(np.abs(got[f] - ref[f])) <= 3e-2 * scale, (world, f)
            assert abs(float(np.mean(got[f] - ref[f]))) <= 1e-3 * scale, (world, f)
        else:
            assert np.array_equal(got[f], ref[f]), (storage, world, f)


def test_copy_plane_rejects_fp16():
    import torch
    with Tau1(19, (32, 8, 4), storage="f16s") as t:
        t.set_geometry(np.zeros((4, 8, 32), np.uint8))
        buf = torch.empty(32 * 8 * 8, dtype=torch.uint8, device="cuda")
        with pytest.raises(Exception):
            t.copy_plane(1, buf, False)
