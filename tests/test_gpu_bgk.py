"""GPU standard BGK (tau = 1, stored populations) vs the oracle's BGK, and
GPU BGK vs GPU Tau1 (Eq. LBMTau1: the two coincide at tau = 1)."""
import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import Tau1, build
from paper_2312_14742_gb300.lbm import LBM_SCHEME_BGK

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def bgk_gpu(q, solid, per, g, storage, nsteps, state=None):
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage=storage, periodic=per, g=g, scheme=LBM_SCHEME_BGK) as t:
        t.set_geometry(solid)
        if state is not None:
            t.set_fields(*state)
        t.step(nsteps)
        out = t.get_fields()
        stats = t.reduce(allow_diverged=True)
    return out, stats


def oracle_bgk(q, solid, per, g, nsteps, state):
    D = oracle.Domain(q, solid, periodic=per, g=g)
    h = D.bgk_init(state, 1.0)
    mom = state
    for _ in range(nsteps):
        h, mom = D.bgk_step(h, 1.0)
    return mom


@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("per", [(1, 1, 1), (1, 0, 1)])
def test_bgk_fp64_matches_oracle(q, per):
    solid, _ = lbm_inputs.sphere_pack(20, 18, 17, 3.0, 0.75, 61)
    st = lbm_inputs.random_fields(solid.shape, 62, 2e-3, 3e-3, solid)
    g = (1e-5, -2e-6, 3e-6)
    out, _ = bgk_gpu(q, solid, per, g, "f64", 40, st)
    ref = oracle_bgk(q, solid, per, g, 40, st)
    umax = max(float(np.max(np.abs(r))) for r in ref[1:])
    assert float(np.max(np.abs(out[0] - ref[0]))) <= 1e-12
    assert max(float(np.max(np.abs(o - r))) for o, r in zip(out[1:], ref[1:])) <= 1e-12 * umax


@pytest.mark.parametrize("q", (19, 27))
def test_bgk_fp32_matches_oracle_1000_steps(q):
    solid, _ = lbm_inputs.sphere_pack(48, 40, 36, 4.0, 0.9, 63)
    g = (1e-5, 0, 0)
    z = [np.zeros(solid.shape) for _ in range(4)]
    out, _ = bgk_gpu(q, solid, (1, 1, 1), g, "f32", 1000)
    D = oracle.Domain(q, solid, periodic=(1, 1, 1), g=g)
    ref = D.tau1_run(z, 1000)  # oracle Tau1 == oracle BGK at tau = 1 (pinned on the CPU)
    umax = max(float(np.max(np.abs(r))) for r in ref[1:])
    assert max(float(np.max(np.abs(o - r))) for o, r in zip(out[1:], ref[1:])) <= 1e-5 * umax


@pytest.mark.parametrize("q", (19, 27))
def test_bgk_equals_tau1_on_gpu(q):
    solid, _ = lbm_inputs.sphere_pack(40, 33, 29, 3.0, 0.8, 64)
    st = lbm_inputs.random_fields(solid.shape, 65, 1e-3, 2e-3, solid)
    g = (2e-5, 0, -1e-5)
    a, sa = bgk_gpu(q, solid, (1, 1, 1), g, "f64", 100, st)
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage="f64", g=g) as t:
        t.set_geometry(solid)
        t.set_fields(*st)
        t.step(100)
        b = t.get_fields()
        sb = t.reduce()
    umax = max(float(np.max(np.abs(x))) for x in b[1:])
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(a[1:], b[1:])) <= 1e-13 * umax
    assert float(np.max(np.abs(a[0] - b[0]))) <= 1e-14
    assert sa["n_fluid"] == sb["n_fluid"]


def test_bgk_rejects_16bit_storage():
    with pytest.raises(Exception):
        Tau1(19, (8, 8, 8), storage="f16s", scheme=LBM_SCHEME_BGK)
