"""Batches: many boxes of different sizes stepped in one persistent launch,
K-step CUDA graphs, admission by device footprint.

Every box of a batch must give exactly what the single-box path gives (FP32
and FP64: same bits), the FP64 oracle's result within 1e-12, and the same
bits alone as in any mix of other boxes admitted and released around it
(all storage formats, 16-bit included: a box's scales and stochastic
rounding depend on its own state and step count only)."""
import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import Batch, Tau1, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def boxes(seed=0):
    """(solid, periodic, g) of boxes with ragged tiles, walls and periodic axes."""
    out = []
    s, _ = lbm_inputs.sphere_pack(32, 32, 32, 4.0, 0.8, lbm_inputs.workload_seed(5, seed))
    out.append((s, (1, 1, 1), (1e-5, 0.0, 0.0)))
    s, _ = lbm_inputs.sphere_pack(48, 40, 36, 3.0, 0.7, lbm_inputs.workload_seed(5, seed + 1))
    s[0] = 1
    s[-1] = 1
    out.append((s, (1, 1, 0), (2e-5, -1e-5, 0.0)))
    out.append((lbm_inputs.channel(20, 50, 17), (1, 1, 0), (1e-5, 0.0, 0.0)))
    s, _ = lbm_inputs.sphere_pack(70, 9, 33, 2.5, 0.75, lbm_inputs.workload_seed(5, seed + 2))
    out.append((s, (1, 1, 1), (0.0, 0.0, 3e-5)))
    return out


def single(q, storage, solid, per, g, steps):
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage=storage, periodic=per, g=g, kernel="tiled") as t:
        t.set_geometry(solid)
        t.step(steps)
        return t.get_fields(), t.reduce()


def variants(q, storage):
    return (0,) if storage == "f64" else (0, 1, 2, 3)


@pytest.mark.parametrize("q", (19, 27))
@pytest.mark.parametrize("storage", ("f32", "f64"))
def test_batch_equals_single_box_bitwise(q, storage):
    """250 steps = two replays of a 100-step graph plus 50 single launches."""
    bx = boxes()
    refs = [single(q, storage, *b, 250) for b in bx]
    for v in variants(q, storage):
        with Batch(q, storage, capacity=8, variant=v, graph_steps=100) as B:
            slots = [B.admit(s, per, g) for s, per, g in bx]
            assert B.live == len(bx)
            B.step(250)
            stats = B.stats(slots)
            for k, slot in enumerate(slots):
                got = B.get_fields(slot)
                for a in range(4):
                    assert np.array_equal(got[a], refs[k][0][a]), (v, k, a)
                assert stats[k]["step"] == 250
                for key in ("mean_ux_superficial", "max_abs_u", "drho_sum", "n_fluid"):
                    assert stats[k][key] == refs[k][1][key], (v, k, key)


@pytest.mark.parametrize("q", (19, 27))
def test_batch_fp64_matches_oracle(q):
    solid, per, g = boxes(3)[1]
    D = oracle.Domain(q, solid, periodic=per, g=g)
    ref = D.tau1_run(D.zero_state(), 60)
    with Batch(q, "f64", capacity=4, graph_steps=25) as B:
        other = B.admit(boxes(3)[0][0], (1, 1, 1), (1e-5, 0, 0))
        slot = B.admit(solid, per, g)
        B.step(60)
        got = B.get_fields(slot)
        assert other is not None
    umax = max(float(np.max(np.abs(ref[a]))) for a in (1, 2, 3))
    assert float(np.max(np.abs(got[0] - ref[0]))) <= 1e-12
    assert max(float(np.max(np.abs(got[a] - ref[a]))) for a in (1, 2, 3)) <= 1e-12 * umax


@pytest.mark.parametrize("storage", ("f32", "f16s", "bf16s"))
def test_same_bits_alone_and_in_a_mix(storage):
    """Box X alone for 300 steps, and inside a batch whose other boxes come and
    go (admitted before and after X, one released mid-run): same bits."""
    q = 19
    bx = boxes(7)
    X = bx[1]
    with Batch(q, storage, capacity=8, graph_steps=64) as A:
        sa = A.admit(*X)
        A.step(300)
        alone = A.get_fields(sa)
        alone_stats = A.stats([sa])[0]
    with Batch(q, storage, capacity=8, graph_steps=64) as B:
        o1 = B.admit(*bx[0])
        o2 = B.admit(*bx[2])
        B.step(37)
        sx = B.admit(*X)
        B.step(100)
        B.release(o1)
        o3 = B.admit(*bx[3])
        B.step(130)
        o4 = B.admit(*boxes(9)[0])
        B.step(70)
        mixed = B.get_fields(sx)
        mixed_stats = B.stats([sx, o2, o3, o4])
    for a in range(4):
        assert np.array_equal(alone[a], mixed[a]), (storage, a)
    assert mixed_stats[0]["step"] == 300 and mixed_stats[1]["step"] == 337
    assert mixed_stats[2]["step"] == 200 and mixed_stats[3]["step"] == 70
    assert mixed_stats[0]["mean_ux_superficial"] == alone_stats["mean_ux_superficial"]


def test_admission_by_footprint_and_capacity():
    bx = boxes(11)
    fa = Batch.footprint("f32", bx[0][0].shape[::-1])
    fb = Batch.footprint("f32", bx[1][0].shape[::-1])
    with Batch(19, "f32", capacity=8, hbm_budget=fa + fb - 1) as B:
        a = B.admit(*bx[0])
        assert a is not None and B.bytes_free == fb - 1
        assert B.admit(*bx[1]) is None  # does not fit now
        B.step(10)
        B.release(a)
        assert B.bytes_free == fa + fb - 1
        b = B.admit(*bx[1])
        assert b is not None
        B.step(5)
        assert B.stats([b])[0]["step"] == 5
    with Batch(19, "f32", capacity=2) as B:
        assert B.admit(*bx[0]) is not None
        assert B.admit(*bx[2]) is not None
        assert B.admit(*bx[3]) is None  # capacity reached
        assert B.live == 2


def test_empty_batch_and_graph_remainders():
    """Steps with no live box do nothing; any split of n steps into graph
    replays and single launches gives the same bits."""
    solid, per, g = boxes(13)[0]
    with Batch(19, "f32", capacity=2, graph_steps=7) as B:
        B.step(5)
        s = B.admit(solid, per, g)
        B.step(3)
        B.step(7)
        B.step(16)
        got = B.get_fields(s)
        assert B.stats([s])[0]["step"] == 26
    ref, _ = single(19, "f32", solid, per, g, 26)
    for a in range(4):
        assert np.array_equal(got[a], ref[a])


def test_fp16_batch_box_permeability_within_one_percent():
    """A porous box with FP16 storage in a batch (scales chosen by the step
    kernel's closing block): permeability averaged over 10 states 50 steps
    apart after 3000 steps, within 1 % of the FP64 oracle's over the same
    window."""
    solid, _ = lbm_inputs.sphere_pack(40, 40, 40, 4.0, 0.6, lbm_inputs.workload_seed(5, 40))
    g = (1e-5, 0.0, 0.0)
    from oracle_steady import oracle_window
    k64 = oracle_window(19, solid, (1, 1, 1), g, 3000)
    with Batch(19, "f16s", capacity=4, graph_steps=100) as B:
        B.admit(*boxes(17)[0])
        s = B.admit(solid, (1, 1, 1), g)
        B.step(3000)
        ks = []
        for _ in range(10):
            B.step(50)
            ks.append(B.stats([s])[0]["permeability"])
    assert abs(np.mean(ks) - k64) <= 1e-2 * abs(k64), (np.mean(ks), k64)


def test_batch_error_paths():
    """Wrong lattice or storage, non-dense layout, a slot that is not live,
    and a negative step count are refused without changing the batch."""
    from paper_2312_14742_gb300 import lbm
    solid = boxes(19)[0][0]
    with Batch(19, "f32", capacity=4) as B:
        s = B.admit(solid, (1, 1, 1), (1e-5, 0, 0))
        for q, st, layout in ((27, "f32", lbm.LBM_DENSE), (19, "f64", lbm.LBM_DENSE), (19, "f32", lbm.LBM_SPARSE)):
            cfg = lbm.box_config(q, solid.shape[::-1], st)
            cfg.layout = layout
            code, slot = lbm.lbm_tau1_batch_admit(B.b, cfg, solid.ctypes.data, 0)
            assert code == lbm.LBM_EINVAL and slot == -1
        assert lbm.lbm_tau1_batch_release(B.b, 3) == lbm.LBM_EINVAL
        assert lbm.lbm_tau1_batch_release(B.b, -1) == lbm.LBM_EINVAL
        assert lbm.lbm_tau1_batch_step(B.b, -1) == lbm.LBM_EINVAL
        assert B.live == 1
        B.step(3)
        B.release(s)
        assert lbm.lbm_tau1_batch_release(B.b, s) == lbm.LBM_EINVAL
        assert B.live == 0
        B.step(5)  # nothing live: no work


def test_poisoned_box_does_not_touch_its_neighbours():
    """A box driven to divergence (g far too large) is reported by stats and
    released; the other box of the batch keeps the bits it has alone."""
    good, per, g = boxes(21)[0]
    bad = boxes(21)[2][0]
    with Batch(19, "f32", capacity=4, graph_steps=50) as A:
        s = A.admit(good, per, g)
        A.step(200)
        alone = A.get_fields(s)
    with Batch(19, "f32", capacity=4, graph_steps=50) as B:
        s = B.admit(good, per, g)
        x = B.admit(bad, (1, 1, 0), (0.2, 0.0, 0.0))
        B.step(200)
        st = B.stats([s, x], allow_diverged=True)
        assert st[0]["nonfinite"] == 0 and st[0]["max_abs_u"] < 0.3
        assert st[1]["nonfinite"] > 0 or st[1]["max_abs_u"] > 0.3
        B.release(x)
        mixed = B.get_fields(s)
    for a, b in zip(alone, mixed):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ("f32", "f16s"))
def test_queued_stats_equal_stats(storage):
    """Statistics queued behind the steps (stats_queue) and taken later
    (stats_wait) equal the synchronous ones of the same moment, whatever is
    queued in between: more steps, the release of a box, an admission."""
    from paper_2312_14742_gb300 import lbm
    bx = boxes(23)
    with Batch(19, storage, capacity=6, graph_steps=50) as B:
        slots = [B.admit(s, per, g) for s, per, g in bx[:3]]
        B.step(150)
        ref = B.stats(slots, allow_diverged=True)
        B.stats_queue(slots)
        assert lbm.lbm_tau1_batch_stats_queue(B.b, 0, None) == lbm.LBM_ESTATE  # one request at a time
        B.step(100)
        B.release(slots[1])
        extra = B.admit(*bx[3])
        got = B.stats_wait(allow_diverged=True)
        assert got == ref
        assert all(r["step"] == 150 for r in got)
        later = B.stats([slots[0], slots[2]], allow_diverged=True)
        assert [r["step"] for r in later] == [250, 250] and later[0] != ref[0]
        assert lbm.lbm_tau1_batch_stats_wait(B.b, None) == lbm.LBM_ESTATE  # nothing queued
        B.stats_queue([slots[0], extra])
        B.step(50)
        got = B.stats_wait(allow_diverged=True)
        assert [r["step"] for r in got] == [250, 0]
