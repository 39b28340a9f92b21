"""The serving loop on the GPU: continuously batched requests against the
plain one-at-a-time server on the same arrivals.

FP32 batched and plain evaluate each sample with the same kernel arithmetic
(a box gives the same bits in a batch as alone), so every request converges
at the same step with the same permeability bits. FP16 storage stays within
1% of the FP32 permeability. A request's answer does not depend on which
other requests shared the batch."""
import pytest

from paper_2312_14742_gb300 import build, serve

pytestmark = pytest.mark.gpu

EDGES = (32, 48, 64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.fixture(scope="module")
def requests():
    reqs = serve.make_requests(10, 20231222 + 5000 + 77, edges=EDGES)
    arr = serve.poisson_arrivals(10, 40.0, 5)
    for r, a in zip(reqs, arr):
        r.arrival = float(a)
    return reqs


@pytest.fixture(scope="module")
def plain(requests):
    res, _ = serve.serve_plain(requests, tol=1e-6, cap=4000)
    return {r.id: r for r in res}


def run_batched(reqs, storage, capacity=8, overlap=True):
    srv = serve.BatchedServer(storage=storage, capacity=capacity, tol=1e-6, cap=4000, overlap=overlap)
    try:
        return {r.id: r for r in srv.run(reqs)}, srv
    finally:
        srv.batch.close()


@pytest.mark.parametrize("overlap", (True, False))
def test_batched_fp32_equals_plain(requests, plain, overlap):
    """With and without host/device overlap (statistics taken while the next
    chunk runs)."""
    got, srv = run_batched(requests, "f32", overlap=overlap)
    assert sorted(got) == sorted(plain)
    for i, r in got.items():
        assert r.status == plain[i].status
        assert r.steps == plain[i].steps, i
        assert r.permeability == plain[i].permeability, i
        assert r.latency > 0
    assert srv.fluid_updates == sum(r.n_fluid * r.steps for r in got.values())


def test_batched_fp16_permeability_within_one_percent(requests, plain):
    got, _ = run_batched(requests, "f16s")
    for i, r in got.items():
        assert r.status in ("converged", "cap")
        assert abs(r.permeability - plain[i].permeability) <= 1e-2 * abs(plain[i].permeability), i


@pytest.mark.parametrize("storage", ("f32", "f16s"))
def test_answer_alone_equals_answer_in_the_mix(requests, storage):
    mixed, _ = run_batched(requests, storage, capacity=4)
    for pick in (0, 7):
        alone = serve.Request(**{**requests[pick].__dict__, "arrival": 0.0})
        res, _ = run_batched([alone], storage)
        r = res[alone.id]
        assert r.steps == mixed[alone.id].steps
        assert r.permeability == mixed[alone.id].permeability
