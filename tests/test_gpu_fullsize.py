"""Parity at the benchmark's full size, in the launch configuration the
benchmark times (256^3 periodic box, overlapping spheres of radius 8 to
porosity 0.9, g_x = 1e-5, FP32 storage, tiled kernel after autotuning).

The oracle cannot run the whole box for many steps, so it evaluates one step
at sampled nodes from the GPU's state (each sample computed one by one), and
properties that hold at any size are checked on the whole box.
"""
import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import Tau1, build

pytestmark = pytest.mark.gpu

N = 256


@pytest.fixture(scope="module")
def medium():
    build.build()
    solid, info = lbm_inputs.sphere_pack(N, N, N, 8.0, 0.9, lbm_inputs.workload_seed(1, 0))
    return solid, info


@pytest.mark.parametrize("q", (19, 27))
def test_fullsize_sampled_one_step(medium, q):
    solid, info = medium
    assert info.porosity <= 0.9
    g = (1e-5, 0.0, 0.0)
    with Tau1(q, (N, N, N), storage="f32", g=g) as t:
        t.set_geometry(solid)
        t.step(10)
        t.autotune(5)
        t.step(19)
        before = t.get_fields()
        s0 = t.reduce()
        t.step(1)
        after = t.get_fields()
        s1 = t.reduce()
    rng = np.random.default_rng(q)
    fluid = np.flatnonzero(solid.reshape(-1) == 0)
    # sampled nodes, with every wall-adjacent kind likely present
    idx = np.sort(rng.choice(fluid, size=20000, replace=False))
    D = oracle.Domain(q, solid, periodic=(1, 1, 1), g=g)
    ref = D.tau1_nodes(before, idx)
    got = np.stack([a.reshape(-1)[idx] for a in after], axis=1)
    umax = float(np.max(np.abs(ref[:, 1:])))
    dmax = float(np.max(np.abs(ref[:, 0])))
    assert np.max(np.abs(got[:, 1:] - ref[:, 1:])) <= 1e-5 * umax
    assert np.max(np.abs(got[:, 0] - ref[:, 0])) <= 1e-5 * dmax + 1e-9
    # solid nodes untouched, mass conserved to FP32 rounding
    assert np.all(after[0][solid != 0] == 0) and np.all(after[1][solid != 0] == 0)
    nf = s1["n_fluid"]
    assert nf == int(fluid.size)
    assert abs(s1["drho_sum"] - s0["drho_sum"]) <= 1e-6 * nf * max(dmax, 1e-6)
    # the reduction of the GPU state equals the oracle's reduction of the same
    # state: both sum in FP64, the oracle sequentially over 15 M nodes, the GPU
    # in a tree, so the sums differ by ~N eps relative at most (~3e-9)
    r = D.reduce(after)
    assert abs(s1["mean_ux_superficial"] - r["mean_ux_superficial"]) <= 1e-8 * abs(r["mean_ux_superficial"])
    assert abs(s1["max_abs_u"] - r["max_abs_u"]) <= 1e-12 * r["max_abs_u"]
