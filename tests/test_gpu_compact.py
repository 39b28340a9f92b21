"""Compact porous layout (dense records, work split by tile column) against
the dense kernels and the oracle.

Every link of a compact step is computed by one of the dense kernels (the
row-pair kernel over a list of tile columns, the one-thread-per-node kernel
over a node list) and each node is written by exactly one of them, so the
compact state equals the dense state bit for bit, whatever the threshold f*
that splits the tile columns. FP64 also matches the oracle to 1e-12, FP32 to
1e-5 of the largest velocity (the tolerances of the dense parity tests)."""
import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import Tau1, build
from paper_2312_14742_gb300.lbm import COMPACT_THRESHOLDS, LBM_COMPACT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def run(q, solid, per, g, storage, steps, state=None, layout=0, kernel="auto", thr=None, pressure=None,
        autotune=False):
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage=storage, periodic=per, g=g, layout=layout, kernel=kernel) as t:
        if thr is not None:
            t.set_compact_threshold(thr)
        t.set_geometry(solid)
        if state is not None:
            t.set_fields(*state)
        if pressure is not None:
            t.set_pressure(*pressure)
        if autotune:
            t.autotune(3)
        t.step(steps)
        info = t.compact_info() if layout == LBM_COMPACT else None
        return t.get_fields(), t.reduce(allow_diverged=True), info


def mixed_medium(nx, ny, nz, seed):
    """Tile columns of every class: a dense sphere pack on the left half
    (fluid fractions near 0.2), an open right half (near 0.9), and one x-y
    tile (x < 32, y < 8) solid through the whole box, so that its tile columns
    have no fluid node."""
    left, _ = lbm_inputs.sphere_pack(nx, ny, nz, 3.0, 0.2, seed)
    right, _ = lbm_inputs.sphere_pack(nx, ny, nz, 3.0, 0.9, seed + 1)
    solid = right.copy()
    solid[:, :, : nx // 2] = left[:, :, : nx // 2]
    solid[:, :8, :32] = 1
    return np.ascontiguousarray(solid)


def assert_same(got, ref, tag):
    for a in range(4):
        assert np.array_equal(got[a], ref[a], equal_nan=True), (tag, a)


@pytest.mark.parametrize("storage", ("f32", "f64", "f16s", "bf16s"))
@pytest.mark.parametrize("q", (19, 27))
def test_compact_bitwise_equals_dense_every_threshold(q, storage):
    """64 x 32 x 50: 2 x 4 tiles of 32 x 8, z chunks of 24, 24 and 2 planes."""
    solid = mixed_medium(64, 32, 50, 7100 + q)
    st = lbm_inputs.random_fields(solid.shape, 7101, 2e-3, 3e-3, solid)
    g = (1e-5, -2e-6, 3e-6)
    per = (1, 1, 1)
    ref, rs, _ = run(q, solid, per, g, storage, 30, st)
    nf = int(np.count_nonzero(solid == 0))
    seen = set()
    for thr in (0.0, 0.3, 0.6, 1.01):
        got, gs, info = run(q, solid, per, g, storage, 30, st, layout=LBM_COMPACT, thr=thr)
        assert_same(got, ref, (q, storage, thr))
        assert gs["n_fluid"] == rs["n_fluid"] == nf
        assert gs["max_abs_u"] == rs["max_abs_u"]
        assert info["tiled_ok"] == 1 and info["tile"] == (32, 8, 24)
        assert info["columns"] == 2 * 4 * 3
        assert info["empty_columns"] == 3
        assert info["tiled_columns"] + info["listed_columns"] + info["empty_columns"] == info["columns"]
        assert info["tiled_fluid"] + info["listed_nodes"] == nf
        seen.add((info["tiled_columns"] > 0, info["listed_columns"] > 0))
        if thr == 0.0:
            assert info["listed_columns"] == 0
        if thr == 1.01:
            assert info["tiled_columns"] == 0 and info["listed_nodes"] == nf
    assert seen == {(True, False), (True, True), (False, True)}


@pytest.mark.parametrize("storage", ("f32", "f64", "bf16s"))
def test_compact_every_variant_bitwise_equals_dense(storage):
    """Every row-pair variant (tile shape, 24- or 32-plane chunks) as the
    compact layout's tile column; a shape whose tile height does not divide
    ny = 48 sends every column to the node list."""
    solid = mixed_medium(64, 48, 70, 7150)
    st = lbm_inputs.random_fields(solid.shape, 7151, 2e-3, 3e-3, solid)
    g = (1e-5, -2e-6, 3e-6)
    ref, _, _ = run(19, solid, (1, 1, 1), g, storage, 20, st)
    nz, ny, nx = solid.shape
    nf = int(np.count_nonzero(solid == 0))
    nv = 2 if storage == "f64" else 8
    for v in range(nv):
        # a fresh handle per variant: the 16-bit stochastic rounding draws on the step count
        with Tau1(19, (nx, ny, nz), storage=storage, g=g, layout=LBM_COMPACT) as t:
            assert t.variant_count == nv
            t.set_variant(v)
            t.set_geometry(solid)
            t.set_fields(*st)
            t.step(20)
            got = t.get_fields()
            info = t.compact_info()
            # switching the variant with a geometry set rebuilds the lists; the state is kept
            t.set_variant((v + 1) % nv)
            assert t.compact_info()["variant"] == (v + 1) % nv
            assert_same(t.get_fields(), got, (storage, v, "kept"))
            assert_same(got, ref, (storage, v))
            assert info["variant"] == v and info["tile"][2] == (24 if v < nv // 2 else 32)
            assert info["tiled_fluid"] + info["listed_nodes"] == nf
            assert info["tiled_ok"] == (1 if 48 % info["tile"][1] == 0 else 0)


@pytest.mark.parametrize("storage", ("f32", "f64"))
@pytest.mark.parametrize("dims,per,phi", [((45, 19, 21), (1, 0, 1), 0.5), ((64, 12, 9), (0, 1, 0), 0.7),
                                          ((32, 16, 1), (1, 1, 1), 0.6)])
def test_compact_ragged_boxes(dims, per, phi, storage):
    """Boxes the tiled kernel cannot take (nx not a multiple of 32, ny not of
    8): every tile column goes to the node list; one plane (nz = 1)."""
    nx, ny, nz = dims
    solid, _ = lbm_inputs.sphere_pack(nx, ny, nz, 3.0, phi, 7200 + nx)
    st = lbm_inputs.random_fields(solid.shape, 7201, 2e-3, 3e-3, solid)
    g = (1e-5, -2e-6, 3e-6)
    ref, _, _ = run(19, solid, per, g, storage, 25, st)
    got, _, info = run(19, solid, per, g, storage, 25, st, layout=LBM_COMPACT)
    assert_same(got, ref, dims)
    assert info["listed_nodes"] + info["tiled_fluid"] == int(np.count_nonzero(solid == 0))
    if nx % 32 or ny % 8:
        assert info["tiled_ok"] == 0 and info["tiled_columns"] == 0


@pytest.mark.parametrize("storage", ("f64", "f32"))
@pytest.mark.parametrize("q", (19, 27))
def test_compact_matches_oracle(q, storage):
    solid = mixed_medium(64, 16, 30, 7300 + q)
    solid[:, :, 0] = 1
    per = (0, 1, 1)
    g = (1e-5, 0, 0)
    steps = 80 if storage == "f64" else 300
    D = oracle.Domain(q, solid, periodic=per, g=g)
    ref = D.tau1_run(D.zero_state(), steps)
    got, _, info = run(q, solid, per, g, storage, steps, layout=LBM_COMPACT, thr=0.5)
    assert info["tiled_columns"] > 0 and info["listed_columns"] > 0
    umax = max(float(np.max(np.abs(ref[a]))) for a in (1, 2, 3))
    dmax = float(np.max(np.abs(ref[0])))
    du = max(float(np.max(np.abs(got[a] - ref[a]))) for a in (1, 2, 3))
    dd = float(np.max(np.abs(got[0] - ref[0])))
    if storage == "f64":
        assert dd <= 1e-12 and du <= 1e-12 * umax, (dd, du)
    else:
        assert du <= 1e-5 * umax and dd <= 1e-5 * dmax + 1e-9, (dd, du)


def test_compact_all_solid_and_single_fluid_node():
    solid = np.ones((30, 16, 32), np.uint8)
    out, s, info = run(19, solid, (1, 1, 1), (1e-5, 0, 0), "f32", 3, layout=LBM_COMPACT)
    assert s["n_fluid"] == 0 and all(np.all(a == 0) for a in out)
    assert info["empty_columns"] == info["columns"] == 2 * 2
    solid[20, 3, 4] = 0
    st = [np.zeros(solid.shape) for _ in range(4)]
    st[1][20, 3, 4] = 1e-3
    out, s, info = run(19, solid, (1, 1, 1), (1e-5, 0, 0), "f64", 1, state=st, layout=LBM_COMPACT)
    assert s["n_fluid"] == 1 and info["listed_nodes"] == 1 and info["tiled_columns"] == 0
    # isolated node: rho' = rho, u' = -(u + g)
    assert abs(out[1][20, 3, 4] + (1e-3 + 1e-5)) <= 1e-18


def test_compact_pressure_faces_and_autotune_equal_dense():
    """Constant-density faces on x (the face kernel runs after the split
    step); the autotune trials leave the state as it was."""
    solid = mixed_medium(64, 32, 26, 7400)
    per = (0, 1, 1)
    bc = (0, 1.01, 0.99)
    ref, _, _ = run(19, solid, per, (0, 0, 0), "f32", 200, pressure=bc)
    got, _, info = run(19, solid, per, (0, 0, 0), "f32", 200, layout=LBM_COMPACT, pressure=bc, autotune=True)
    assert_same(got, ref, "pressure")
    assert info["threshold"] in COMPACT_THRESHOLDS


def test_compact_threshold_rejected_out_of_range():
    from paper_2312_14742_gb300.lbm import LbmError
    with Tau1(19, (32, 8, 4), layout=LBM_COMPACT) as t:
        with pytest.raises(LbmError):
            t.set_compact_threshold(1.5)
        with pytest.raises(LbmError):
            t.set_compact_threshold(-0.1)
    with Tau1(19, (32, 8, 4)) as t:
        with pytest.raises(LbmError):
            t.set_compact_threshold(0.3)


@pytest.mark.parametrize("dims,per", [((1, 1, 1), (1, 1, 1)), ((2, 3, 1), (1, 0, 1)), ((5, 1, 7), (0, 1, 1)),
                                      ((1, 9, 4), (1, 1, 0)), ((33, 2, 3), (1, 1, 1))])
@pytest.mark.parametrize("storage", ("f32", "f64"))
def test_compact_degenerate_boxes(dims, per, storage):
    """Axes one or two nodes long (the node-list kernel's division by nx and
    nx ny, and its wrap of an axis onto itself), against the dense kernels."""
    nx, ny, nz = dims
    solid = lbm_inputs.random_mask(nx, ny, nz, 0.2, 7500 + nx * 7 + ny)
    st = lbm_inputs.random_fields(solid.shape, 7501, 2e-3, 3e-3, solid)
    g = (1e-5, -2e-6, 3e-6)
    ref, _, _ = run(19, solid, per, g, storage, 12, st, kernel="simple")
    got, _, info = run(19, solid, per, g, storage, 12, st, layout=LBM_COMPACT)
    assert_same(got, ref, dims)
    assert info["tiled_columns"] == 0 and info["listed_nodes"] == int(np.count_nonzero(solid == 0))


@pytest.mark.parametrize("q", (19, 27))
def test_compact_pressure_faces_match_oracle(q):
    """Constant-density faces on z over a compact split box (tile columns of
    both kinds), FP64 against the oracle."""
    solid = mixed_medium(64, 16, 20, 7600 + q)
    per = (1, 1, 0)
    bc = (2, 1.01, 0.99)
    D = oracle.Domain(q, solid, periodic=per, pressure=bc)
    ref = D.tau1_run(D.zero_state(), 60)
    got, _, info = run(q, solid, per, (0, 0, 0), "f64", 60, layout=LBM_COMPACT, thr=0.5, pressure=bc)
    assert info["tiled_columns"] > 0 and info["listed_columns"] > 0
    umax = max(float(np.max(np.abs(ref[a]))) for a in (1, 2, 3))
    assert float(np.max(np.abs(got[0] - ref[0]))) <= 1e-12
    assert max(float(np.max(np.abs(got[a] - ref[a]))) for a in (1, 2, 3)) <= 1e-12 * umax
