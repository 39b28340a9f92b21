"""CUDA Tau1 path vs the FP64 oracle, through the C ABI.

Tolerances (written per test):
  FP64 storage: |drho_gpu - drho_orc| <= 1e-12 and |u_gpu - u_orc| <= 1e-12 max|u_orc|
                (the paper's FP64 agreement between two implementations).
  FP32 storage: |u_gpu - u_orc| <= 1e-5 max|u_orc| after 1000 steps (the FP32 bar);
                drho is compared at 1e-5 of max|drho_orc| plus 1e-9.
"""
import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import Tau1, build

pytestmark = pytest.mark.gpu

KERNELS = ("simple", "tiled")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def gpu_run(q, solid, periodic, g, storage, nsteps, state=None, kernel="auto"):
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage=storage, periodic=periodic, g=g, kernel=kernel) as t:
        t.set_geometry(solid)
        if state is not None:
            t.set_fields(*state)
        t.step(nsteps)
        out = t.get_fields()
        stats = t.reduce(allow_diverged=True)
    return out, stats


def assert_close_fp64(out, ref, tag=""):
    umax = max(float(np.max(np.abs(ref[a]))) for a in (1, 2, 3))
    dd = float(np.max(np.abs(out[0] - ref[0])))
    du = max(float(np.max(np.abs(out[a] - ref[a]))) for a in (1, 2, 3))
    assert dd <= 1e-12, (tag, dd)
    assert du <= 1e-12 * umax, (tag, du, umax)


def assert_close_fp32(out, ref, tag=""):
    umax = max(float(np.max(np.abs(ref[a]))) for a in (1, 2, 3))
    dmax = float(np.max(np.abs(ref[0])))
    du = max(float(np.max(np.abs(out[a] - ref[a]))) for a in (1, 2, 3))
    dd = float(np.max(np.abs(out[0] - ref[0])))
    assert du <= 1e-5 * umax, (tag, du, umax)
    assert dd <= 1e-5 * dmax + 1e-9, (tag, dd, dmax)


def kernel_available(kernel, q, storage):
    if kernel == "simple":
        return True
    try:
        Tau1(q, (8, 8, 8), storage=storage, kernel=kernel).close()
        return True
    except Exception:
        return False


# ---------------------------------------------------------------------------
# the Poiseuille channel (32^3, walls z = 0 and 31, g_x = 1e-6, 1000 steps, FP64)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("kernel", KERNELS)
def test_poiseuille_channel_fp64(q, kernel):
    if not kernel_available(kernel, q, "f64"):
        pytest.skip(f"{kernel} kernel not built for f64")
    g = 1e-6
    solid = lbm_inputs.channel(32, 32, 32)
    out, stats = gpu_run(q, solid, (1, 1, 0), (g, 0, 0), "f64", 1000, kernel=kernel)
    D = oracle.Domain(q, solid, periodic=(1, 1, 0), g=(g, 0, 0))
    ref = D.tau1_run(D.zero_state(), 1000)
    assert_close_fp64(out, ref, f"D3Q{q} {kernel}")
    # every column equal and u_y = u_z = 0 to rounding
    ux = out[1]
    assert np.max(np.abs(ux - ux[:, :1, :1])) <= 1e-13 * np.max(np.abs(ux))
    assert np.max(np.abs(out[2])) < 1e-17 and np.max(np.abs(out[3])) < 1e-17
    r = D.reduce(ref)
    assert stats["n_fluid"] == r["n_fluid"] == 32 * 32 * 30
    assert abs(stats["mean_ux_superficial"] - r["mean_ux_superficial"]) <= 1e-12 * abs(r["mean_ux_superficial"])


# ---------------------------------------------------------------------------
# porous media, random initial state, ragged sizes, mixed periodicity (FP64)
# ---------------------------------------------------------------------------

CASES = [
    ((20, 18, 17), (1, 1, 1), 3.0, 0.75),
    ((33, 9, 12), (1, 0, 1), 2.5, 0.7),
    ((40, 37, 5), (0, 1, 1), 4.0, 0.85),
    ((7, 70, 11), (1, 1, 0), 2.0, 0.6),
]


@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_porous_random_state_fp64(q, kernel, case):
    if not kernel_available(kernel, q, "f64"):
        pytest.skip(f"{kernel} kernel not built for f64")
    (nx, ny, nz), per, r, phi = CASES[case]
    solid, _ = lbm_inputs.sphere_pack(nx, ny, nz, r, phi, lbm_inputs.workload_seed(7, case))
    st = lbm_inputs.random_fields(solid.shape, 50 + case, 2e-3, 3e-3, solid)
    g = (1e-5, -3e-6, 2e-6)
    out, _ = gpu_run(q, solid, per, g, "f64", 60, state=st, kernel=kernel)
    ref = oracle.Domain(q, solid, periodic=per, g=g).tau1_run(st, 60)
    assert_close_fp64(out, ref, f"D3Q{q} {kernel} case{case}")


# ---------------------------------------------------------------------------
# FP32: porous box of the 256^3 workload's kind at 64^3, 1000 steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("kernel", KERNELS)
def test_porous_fp32_1000_steps(q, kernel):
    if not kernel_available(kernel, q, "f32"):
        pytest.skip(f"{kernel} kernel not built for f32")
    solid, info = lbm_inputs.sphere_pack(64, 64, 64, 4.0, 0.9, lbm_inputs.workload_seed(1, 7))
    g = (1e-5, 0, 0)
    out, stats = gpu_run(q, solid, (1, 1, 1), g, "f32", 1000, kernel=kernel)
    D = oracle.Domain(q, solid, periodic=(1, 1, 1), g=g)
    ref = D.tau1_run(D.zero_state(), 1000)
    assert_close_fp32(out, ref, f"D3Q{q} {kernel}")
    r = D.reduce(ref)
    assert abs(stats["permeability"] - r["permeability"]) <= 1e-4 * abs(r["permeability"])


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 5), (1, 7, 1), (65, 1, 3)])
def test_tiny_and_degenerate_boxes(kernel, dims):
    if not kernel_available(kernel, 19, "f64"):
        pytest.skip("tiled kernel not built")
    nx, ny, nz = dims
    solid = np.zeros((nz, ny, nx), np.uint8)
    st = lbm_inputs.random_fields(solid.shape, 77, 1e-3, 2e-3, None)
    for q in (19, 27):
        for per in ((1, 1, 1), (0, 0, 0), (1, 0, 1)):
            g = (2e-5, 1e-5, -1e-5)
            out, _ = gpu_run(q, solid, per, g, "f64", 7, state=st, kernel=kernel)
            ref = oracle.Domain(q, solid, periodic=per, g=g).tau1_run(st, 7)
            assert_close_fp64(out, ref, f"{dims} {per} D3Q{q}")


@pytest.mark.parametrize("kernel", KERNELS)
def test_all_solid_and_isolated_node(kernel):
    if not kernel_available(kernel, 27, "f32"):
        pytest.skip("tiled kernel not built")
    solid = np.ones((6, 5, 4), np.uint8)
    out, stats = gpu_run(27, solid, (1, 1, 1), (1e-5, 0, 0), "f32", 5, kernel=kernel)
    assert stats["n_fluid"] == 0 and all(np.count_nonzero(a) == 0 for a in out)
    solid[3, 2, 1] = 0
    st = [np.zeros(solid.shape) for _ in range(4)]
    st[0][3, 2, 1], st[1][3, 2, 1], st[2][3, 2, 1] = 0.01, 0.02, -0.01
    g = (1e-4, 2e-4, 0)
    out, _ = gpu_run(19, solid, (1, 1, 1), g, "f64", 1, state=st, kernel=kernel)
    assert abs(out[0][3, 2, 1] - 0.01) < 1e-16
    assert abs(out[1][3, 2, 1] + (0.02 + 1e-4)) < 1e-16
    assert abs(out[2][3, 2, 1] + (-0.01 + 2e-4)) < 1e-16


@pytest.mark.parametrize("kernel", KERNELS)
def test_uniform_acceleration_fp32(kernel):
    if not kernel_available(kernel, 19, "f32"):
        pytest.skip("tiled kernel not built")
    solid = np.zeros((16, 24, 40), np.uint8)
    g = (1e-5, -2e-5, 0.0)
    out, stats = gpu_run(19, solid, (1, 1, 1), g, "f32", 100, kernel=kernel)
    # FP32 rounding of u + g, 100 times: bound at the FP32 bar of 1e-5 relative
    assert np.max(np.abs(out[1] - 100 * g[0])) <= 1e-5 * 100 * abs(g[0])
    assert np.max(np.abs(out[2] - 100 * g[1])) <= 1e-5 * 100 * abs(g[1])
    assert np.max(np.abs(out[0])) <= 1e-9


# ---------------------------------------------------------------------------
# reductions, determinism, state round trip
# ---------------------------------------------------------------------------

def test_reduce_matches_oracle_and_is_deterministic():
    solid, _ = lbm_inputs.sphere_pack(48, 40, 36, 3.0, 0.7, 99)
    st = lbm_inputs.random_fields(solid.shape, 98, 1e-3, 1e-3, solid)
    g = (3e-5, 0, 0)
    nz, ny, nx = solid.shape
    with Tau1(19, (nx, ny, nz), storage="f64", g=g) as t:
        t.set_geometry(solid)
        t.set_fields(*st)
        a = t.reduce()
        b = t.reduce()
        back = t.get_fields()
    assert a == b
    r = oracle.Domain(19, solid, g=g).reduce(st)
    assert a["n_fluid"] == r["n_fluid"]
    assert abs(a["mass"] - r["mass"]) <= 1e-12 * r["mass"]
    assert abs(a["mean_ux_superficial"] - r["mean_ux_superficial"]) <= 1e-12 * abs(r["mean_ux_superficial"])
    assert abs(a["max_abs_u"] - r["max_abs_u"]) <= 1e-15
    assert abs(a["permeability"] - r["permeability"]) <= 1e-12 * abs(r["permeability"])
    for x, y in zip(back, st):
        assert np.array_equal(x, y)


def test_runs_are_bitwise_reproducible():
    solid, _ = lbm_inputs.sphere_pack(64, 48, 40, 4.0, 0.8, 5)
    a, sa = gpu_run(27, solid, (1, 1, 1), (1e-5, 0, 0), "f32", 50)
    b, sb = gpu_run(27, solid, (1, 1, 1), (1e-5, 0, 0), "f32", 50)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert sa == sb


def test_divergence_is_reported_not_trapped():
    solid = np.zeros((8, 8, 8), np.uint8)
    st = [np.zeros(solid.shape) for _ in range(4)]
    st[1][:] = 0.5  # |u| > 0.3: reported as diverged by the reduction
    nz, ny, nx = solid.shape
    with Tau1(19, (nx, ny, nz), storage="f32") as t:
        t.set_geometry(solid)
        t.set_fields(*st)
        d = t.reduce(allow_diverged=True)
        assert d.get("diverged")
        t.step(3)
        t.synchronize()


# ---------------------------------------------------------------------------
# kernel cross-checks: the tiled kernel (every tile-shape variant) equals the
# one-thread-per-node kernel bit for bit (the same per-lane IEEE operations
# in the same order); autotuning leaves the state alone
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ("f32", "f64", "f16s", "bf16s"))
@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("dims,per", [((64, 40, 33), (1, 1, 1)), ((45, 19, 21), (1, 0, 1)), ((7, 70, 9), (0, 1, 0)),
                                      ((64, 48, 40), (1, 0, 1)), ((96, 32, 20), (0, 1, 1))])
def test_tiled_bitwise_equals_simple(q, dims, per, storage):
    """Boxes with full tiles (nx a multiple of 32, ny of the tile height) run the
    staged (TMA) form of the tiled kernel, the others the register form."""
    nx, ny, nz = dims
    solid, _ = lbm_inputs.sphere_pack(nx, ny, nz, 3.0, 0.8, 4242 + nx)
    st = lbm_inputs.random_fields(solid.shape, 17, 2e-3, 3e-3, solid)
    g = (1e-5, 2e-6, -3e-6)
    ref, _ = gpu_run(q, solid, per, g, storage, 25, state=st, kernel="simple")
    with Tau1(q, dims, storage=storage, periodic=per, g=g, kernel="tiled") as t:
        nv = t.variant_count
    assert nv >= 1
    for v in range(nv):
        with Tau1(q, dims, storage=storage, periodic=per, g=g, kernel="tiled") as t:
            t.set_geometry(solid)
            t.set_fields(*st)
            t.set_variant(v)
            t.step(25)
            out = t.get_fields()
        for a in range(4):
            assert np.array_equal(out[a], ref[a]), (q, dims, storage, v, a)


def test_autotune_keeps_state():
    solid, _ = lbm_inputs.sphere_pack(96, 64, 48, 5.0, 0.85, 77)
    st = lbm_inputs.random_fields(solid.shape, 78, 1e-3, 1e-3, solid)
    nz, ny, nx = solid.shape
    with Tau1(19, (nx, ny, nz), storage="f32", g=(1e-5, 0, 0)) as t:
        t.set_geometry(solid)
        t.set_fields(*st)
        t.step(3)
        before = t.get_fields()
        v, ms = t.autotune(5)
        assert 0 <= v < t.variant_count and ms > 0
        after = t.get_fields()
        t.step(2)
        a = t.get_fields()
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    ref, _ = gpu_run(19, solid, (1, 1, 1), (1e-5, 0, 0), "f32", 5, state=st, kernel="simple")
    for x, y in zip(a, ref):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("storage", ("f64", "f32"))
def test_channel_t1000_matches_stored_oracle(q, storage):
    """The 32^3 Poiseuille channel at t = 1000 against the oracle's stored
    column (tests/golden/channel_t1000.json), on the full 32^3 box."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "channel_t1000.json")) as f:
        gold = json.load(f)
    solid = lbm_inputs.channel(32, 32, 32)
    out, _ = gpu_run(q, solid, (1, 1, 0), (gold["g"], 0, 0), storage, gold["steps"])
    ref_u = np.array(gold[f"D3Q{q}"]["ux"])
    ref_d = np.array(gold[f"D3Q{q}"]["drho"])
    tol = 1e-12 if storage == "f64" else 1e-5
    umax = np.max(np.abs(ref_u))
    assert np.max(np.abs(out[1] - ref_u[:, None, None])) <= tol * umax
    assert np.max(np.abs(out[0] - ref_d[:, None, None])) <= (1e-12 if storage == "f64" else 1e-9)
    assert np.max(np.abs(out[2])) <= tol * umax and np.max(np.abs(out[3])) <= tol * umax


def test_autotune_cache(tmp_path):
    """With a cache file set, the first autotune times the variants and
    records its choice; a later handle with the same key takes it from the
    file without launching trials. Entries of other keys are kept."""
    import json
    from paper_2312_14742_gb300 import lbm
    path = tmp_path / "tune.json"
    lbm.lbm_tau1_set_tune_cache(str(path))
    try:
        solid, _ = lbm_inputs.sphere_pack(64, 48, 40, 4.0, 0.8, 5150)
        nz, ny, nx = solid.shape
        with Tau1(19, (nx, ny, nz), storage="f32", g=(1e-5, 0, 0)) as t:
            t.set_geometry(solid)
            v, ms = t.autotune(3)
        entries = json.loads(path.read_text())["entries"]
        (key, rec), = entries.items()
        assert "/D3Q19/F32/dense/n2^17/full" in key and rec["variant"] == v
        with Tau1(19, (nx, ny, nz), storage="f32", g=(1e-5, 0, 0)) as t:
            t.set_geometry(solid)
            n0 = t.launch_count
            v2, ms2 = t.autotune(3)
            assert t.launch_count == n0 and v2 == v and ms2 == pytest.approx(rec["ms_per_step"], rel=1e-5)
        with Tau1(27, (nx, ny, nz), storage="f32", g=(1e-5, 0, 0)) as t:
            t.set_geometry(solid)
            t.autotune(2)
        entries = json.loads(path.read_text())["entries"]
        assert len(entries) == 2 and entries[key]["variant"] == v
    finally:
        lbm.lbm_tau1_set_tune_cache(None)


@pytest.mark.parametrize("storage", ("f32", "f64"))
def test_checkpoint_resume_is_bitwise(storage):
    """get_fields / set_fields are the checkpoint: stepping 30 + 20 across a
    restore into a fresh handle equals 50 uninterrupted steps, bit for bit."""
    solid, _ = lbm_inputs.sphere_pack(40, 24, 18, 3.0, 0.75, 6161)
    nz, ny, nx = solid.shape
    g = (1e-5, -3e-6, 0.0)
    ref, _ = gpu_run(19, solid, (1, 1, 1), g, storage, 50)
    with Tau1(19, (nx, ny, nz), storage=storage, g=g) as t:
        t.set_geometry(solid)
        t.step(30)
        ckpt = t.get_fields()
    with Tau1(19, (nx, ny, nz), storage=storage, g=g) as t:
        t.set_geometry(solid)
        t.set_fields(*ckpt)
        t.step(20)
        got = t.get_fields()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_get_fields_into_pinned_host_arrays():
    """Page-locked host arrays are written by the export kernel directly; the
    values equal those of the staged path into ordinary host arrays."""
    import torch

    solid, _ = lbm_inputs.sphere_pack(40, 24, 18, 3.0, 0.75, 6262)
    nz, ny, nx = solid.shape
    for storage in ("f32", "f16s"):
        with Tau1(19, (nx, ny, nz), storage=storage, g=(1e-5, 2e-6, 0.0)) as t:
            t.set_geometry(solid)
            t.step(30)
            ref = t.get_fields()
            outs = [torch.full((solid.size,), 7.0, dtype=torch.float64).pin_memory() for _ in range(4)]
            from paper_2312_14742_gb300 import lbm as L
            assert L.lbm_tau1_get_fields(t.h, *[o.data_ptr() for o in outs], 0) == 0
        for a in range(4):
            assert np.array_equal(outs[a].numpy().reshape(solid.shape), ref[a]), (storage, a)
