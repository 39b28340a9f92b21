"""Sparse layout (fluid list + int32 neighbour table) against the dense
kernels and the oracle.

The sparse step evaluates every link with the dense kernels' operations in
their order, so FP32 and FP64 results equal the dense one-thread-per-node
kernel bit for bit; FP64 also matches the oracle to 1e-12."""
import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import Tau1, build
from paper_2312_14742_gb300.lbm import LBM_SPARSE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def run(q, solid, per, g, storage, steps, state=None, layout=0, kernel="simple"):
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage=storage, periodic=per, g=g, layout=layout, kernel=kernel) as t:
        t.set_geometry(solid)
        if state is not None:
            t.set_fields(*state)
        t.step(steps)
        return t.get_fields(), t.reduce(allow_diverged=True)


CASES = [((45, 19, 21), (1, 0, 1), 0.8), ((64, 40, 33), (1, 1, 1), 0.5), ((7, 70, 9), (0, 1, 0), 0.9),
         ((33, 33, 33), (1, 1, 1), 0.3)]


@pytest.mark.parametrize("storage", ("f32", "f64"))
@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("dims,per,phi", CASES)
def test_sparse_bitwise_equals_dense(q, dims, per, phi, storage):
    nx, ny, nz = dims
    solid, _ = lbm_inputs.sphere_pack(nx, ny, nz, 3.0, phi, 9000 + nx)
    st = lbm_inputs.random_fields(solid.shape, 23, 2e-3, 3e-3, solid)
    g = (1e-5, -2e-6, 3e-6)
    ref, rs = run(q, solid, per, g, storage, 30, st)
    got, gs = run(q, solid, per, g, storage, 30, st, layout=LBM_SPARSE)
    for a in range(4):
        assert np.array_equal(got[a], ref[a]), (q, dims, storage, a)
    assert gs["n_fluid"] == rs["n_fluid"] == int(np.count_nonzero(solid == 0))
    assert gs["n_nodes"] == rs["n_nodes"]
    assert gs["max_abs_u"] == rs["max_abs_u"]
    assert abs(gs["mean_ux_superficial"] - rs["mean_ux_superficial"]) <= 1e-13 * abs(rs["mean_ux_superficial"])


@pytest.mark.parametrize("q", (19, 27))
def test_sparse_fp64_matches_oracle(q):
    solid, _ = lbm_inputs.sphere_pack(24, 20, 18, 3.0, 0.6, 31337)
    solid[:, :, 0] = 1
    per = (0, 1, 1)
    g = (1e-5, 0, 0)
    D = oracle.Domain(q, solid, periodic=per, g=g)
    ref = D.tau1_run(D.zero_state(), 80)
    got, _ = run(q, solid, per, g, "f64", 80, layout=LBM_SPARSE)
    umax = max(float(np.max(np.abs(ref[a]))) for a in (1, 2, 3))
    assert float(np.max(np.abs(got[0] - ref[0]))) <= 1e-12
    assert max(float(np.max(np.abs(got[a] - ref[a]))) for a in (1, 2, 3)) <= 1e-12 * umax


def test_sparse_all_solid_and_single_fluid_node():
    solid = np.ones((5, 6, 7), np.uint8)
    out, s = run(19, solid, (1, 1, 1), (1e-5, 0, 0), "f32", 3, layout=LBM_SPARSE)
    assert s["n_fluid"] == 0 and all(np.all(a == 0) for a in out)
    solid[2, 3, 4] = 0
    st = [np.zeros(solid.shape) for _ in range(4)]
    st[1][2, 3, 4] = 1e-3
    out, s = run(19, solid, (1, 1, 1), (1e-5, 0, 0), "f64", 1, state=st, layout=LBM_SPARSE)
    # isolated node: rho' = rho, u' = -(u + g)
    assert s["n_fluid"] == 1
    assert abs(out[1][2, 3, 4] + (1e-3 + 1e-5)) <= 1e-18


@pytest.mark.parametrize("storage", ("f16s", "bf16s"))
def test_sparse_16bit_permeability(storage):
    """Sparse layout with 16-bit storage: permeability averaged over 10 states
    50 steps apart after 1500 steps, within 1 % of the FP64 oracle's over the
    same window."""
    solid, _ = lbm_inputs.sphere_pack(40, 40, 40, 4.0, 0.5, lbm_inputs.workload_seed(3, 40))
    g = (1e-5, 0, 0)
    from oracle_steady import oracle_window
    k64 = oracle_window(19, solid, (1, 1, 1), g, 1500)
    with Tau1(19, (40, 40, 40), storage=storage, g=g, layout=LBM_SPARSE) as t:
        t.set_geometry(solid)
        t.step(1500)
        ks = []
        for _ in range(10):
            t.step(50)
            ks.append(t.reduce()["permeability"])
    assert abs(np.mean(ks) - k64) <= 1e-2 * abs(k64)
