"""Failure detection without a GPU fault.

A staged copy that never lands must end its bounded wait, count a timeout on
the device and reach the host as LBM_ETIMEOUT, with the context still usable.
lbm_tau1_selftest_timeout makes exactly that happen on purpose: one warp
waits, with the step kernels' bounded wait, on an mbarrier phase that nothing
completes (a flag nobody sets), and counts the timeout in the handle's (or
the batch's) counter. The tests check that every reporting call surfaces it
once and that stepping goes on afterwards."""
import numpy as np
import pytest

from paper_2312_14742_gb300 import Batch, Tau1, build, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def expect_timeout(call):
    with pytest.raises(lbm.LbmError) as e:
        call()
    assert e.value.status == lbm.LBM_ETIMEOUT, e.value


def test_single_box_reports_a_wait_that_ran_out():
    with Tau1(19, (32, 16, 8)) as t:
        t.set_geometry(np.zeros((8, 16, 32), np.uint8))
        t.step(3)
        t.synchronize()
        assert lbm.lbm_tau1_selftest_timeout(t.h) == lbm.LBM_OK
        expect_timeout(t.synchronize)
        t.synchronize()  # reported once, then cleared
        t.step(5)
        assert t.reduce()["step"] == 8
        assert lbm.lbm_tau1_selftest_timeout(t.h) == lbm.LBM_OK
        expect_timeout(t.reduce)
        assert t.reduce()["step"] == 8


def test_batch_reports_a_wait_that_ran_out():
    solid = np.zeros((16, 16, 32), np.uint8)
    with Batch(19, "f32", capacity=2, graph_steps=10) as B:
        s = B.admit(solid, (1, 1, 1), (1e-5, 0.0, 0.0))
        B.step(10)
        assert lbm.lbm_tau1_batch_selftest_timeout(B.b) == lbm.LBM_OK
        expect_timeout(B.synchronize)
        B.synchronize()
        assert lbm.lbm_tau1_batch_selftest_timeout(B.b) == lbm.LBM_OK
        B.stats_queue([s])
        expect_timeout(B.stats_wait)
        B.step(10)
        assert B.stats([s])[0]["step"] == 20
