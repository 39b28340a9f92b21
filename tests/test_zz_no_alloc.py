"""lbm_tau1_reduce_noalloc: the reduction for callers that cannot allocate
device memory (a caller working from its own fixed device arena, or inside a
framework whose allocator must account for all device memory). It must give
what the handle-based lbm_tau1_reduce gives for the same state, call after
call, although its scratch is one static device array shared by all calls.

Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import lbm_inputs
from paper_2312_14742_gb300 import Tau1, build, lbm

pytestmark = pytest.mark.gpu

DTYPES = {"f64": "float64", "f32": "float32"}


def _state(dims, seed):
    nx, ny, nz = dims
    solid, _ = lbm_inputs.sphere_pack(nx, ny, nz, 3.0, 0.75, seed)
    st = lbm_inputs.random_fields(solid.shape, seed + 1, 1e-3, 2e-3, solid)
    return solid, st


def _handle_stats(dims, storage, solid, st, g):
    with Tau1(19, dims, storage=storage, g=g) as t:
        t.set_geometry(solid)
        t.set_fields(*st)
        return t.reduce()


def _noalloc(torch, storage, solid, st, g):
    dt = getattr(torch, DTYPES[storage])
    dev = torch.device("cuda", 0)
    fields = [torch.from_numpy(np.ascontiguousarray(a)).to(dev).to(dt) for a in st]
    mask = torch.from_numpy(np.ascontiguousarray(solid)).to(dev)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
    gg = (ctypes.c_double * 3)(*g)
    stream = torch.cuda.current_stream(dev)
    rc = lbm.lbm_tau1_reduce_noalloc(lbm.STORAGE[storage], solid.size, *[f.data_ptr() for f in fields], None,
                                     mask.data_ptr(), gg, out.data_ptr(), stream.cuda_stream)
    assert rc == lbm.LBM_OK, lbm.lbm_tau1_noalloc_last_error()
    torch.cuda.synchronize(dev)
    return out.cpu().numpy()


def _check(raw, ref, n):
    assert int(raw[0]) == ref["n_fluid"]
    assert int(raw[6]) == ref["nonfinite"] == 0
    assert abs(raw[1] - ref["drho_sum"]) <= 1e-12 * max(1.0, abs(ref["drho_sum"]))
    assert abs(raw[2] / n - ref["mean_ux_superficial"]) <= 1e-12 * abs(ref["mean_ux_superficial"])
    for a in range(3):
        want = ref["mean_u_fluid"][a]
        assert abs(raw[2 + a] / ref["n_fluid"] - want) <= 1e-12 * abs(want)
    assert abs(raw[5] - ref["max_abs_u"]) <= 1e-12 * ref["max_abs_u"]


def test_noalloc_matches_reduce_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    build.build()
    lbm.load()
    g = (2e-5, -1e-5, 0.0)
    cases = [((48, 40, 36), "f64", 301), ((20, 18, 17), "f32", 302)]
    refs = []
    for dims, storage, seed in cases:
        solid, st = _state(dims, seed)
        refs.append((dims, storage, solid, st, _handle_stats(dims, storage, solid, st, g)))
    # two calls in a row: the larger box, then the smaller one (which leaves
    # rows of the first call untouched in the shared scratch), then repeat
    for _ in range(2):
        for dims, storage, solid, st, ref in refs:
            raw = _noalloc(torch, storage, solid, st, g)
            _check(raw, ref, solid.size)


def test_noalloc_16bit_with_scales_matches_oracle():
    """16-bit storage with non-unit per-field scales (value = stored *
    inv_scale): the noalloc reduction of the stored arrays equals the FP64
    oracle's reduction of the dequantised state (exact in FP64, since the
    scales are powers of two), on two calls in a row for each format."""
    torch = pytest.importorskip("torch")
    import oracle
    assert torch.cuda.is_available()
    build.build()
    lbm.load()
    dev = torch.device("cuda", 0)
    g = (2e-5, -1e-5, 3e-6)
    dims = (40, 36, 30)
    solid, st = _state(dims, 303)
    ref_dom = oracle.Domain(19, solid, g=g)
    for storage, np16, scale in (("f16s", np.float16, (2.0 ** 10, 2.0 ** 12, 2.0 ** 11, 2.0 ** 13)),
                                 ("bf16s", None, (2.0 ** 4, 2.0 ** -2, 2.0 ** 6, 2.0 ** 3))):
        if np16 is not None:
            stored = [np.ascontiguousarray((a * s).astype(np16)) for a, s in zip(st, scale)]
            deq = [b.astype(np.float64) / s for b, s in zip(stored, scale)]
            tens = [torch.from_numpy(b.view(np.int16)) for b in stored]
        else:
            # BF16: round the FP32 value to the nearest bfloat16 with torch, on the CPU
            tb = [torch.from_numpy(a * s).to(torch.float32).to(torch.bfloat16) for a, s in zip(st, scale)]
            deq = [b.to(torch.float64).numpy() / s for b, s in zip(tb, scale)]
            tens = [b.view(torch.int16) for b in tb]
        fields = [t.contiguous().to(dev) for t in tens]
        mask = torch.from_numpy(np.ascontiguousarray(solid)).to(dev)
        inv = (ctypes.c_float * 4)(*[1.0 / s for s in scale])
        gg = (ctypes.c_double * 3)(*g)
        ref = ref_dom.reduce(deq)
        nf = ref["n_fluid"]
        for _ in range(2):
            out = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
            rc = lbm.lbm_tau1_reduce_noalloc(lbm.STORAGE[storage], solid.size, *[f.data_ptr() for f in fields], inv,
                                             mask.data_ptr(), gg, out.data_ptr(),
                                             torch.cuda.current_stream(dev).cuda_stream)
            assert rc == lbm.LBM_OK, lbm.lbm_tau1_noalloc_last_error()
            torch.cuda.synchronize(dev)
            raw = out.cpu().numpy()
            assert int(raw[0]) == nf and int(raw[6]) == 0
            assert abs(raw[1] - (ref["mass"] - nf)) <= 1e-12 * max(1.0, abs(ref["mass"] - nf))
            assert abs(raw[2] / solid.size - ref["mean_ux_superficial"]) <= 1e-12 * abs(ref["mean_ux_superficial"])
            for a in range(3):
                # the means cancel (values of both signs): bound the summation
                # error by the size of the terms, not of their mean
                want = ref["mean_u_fluid"][a]
                scale_u = max(abs(want), float(np.mean(np.abs(deq[1 + a][solid == 0]))))
                assert abs(raw[2 + a] / nf - want) <= 1e-12 * scale_u, (storage, a)
            assert abs(raw[5] - ref["max_abs_u"]) <= 1e-12 * ref["max_abs_u"]


def test_noalloc_rejects_bad_sizes():
    build.build()
    lbm.load()
    gg = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    big = (1 << 33) + 1
    rc = lbm.lbm_tau1_reduce_noalloc(lbm.LBM_F32, big, 8, 8, 8, 8, None, 8, gg, 8, None)
    assert rc == lbm.LBM_EINVAL
    assert "LBM_TAU1_NOALLOC_MAX_NODES" in lbm.lbm_tau1_noalloc_last_error()
    rc = lbm.lbm_tau1_reduce_noalloc(lbm.LBM_F32, 0, 8, 8, 8, 8, None, 8, gg, 8, None)
    assert rc == lbm.LBM_EINVAL
