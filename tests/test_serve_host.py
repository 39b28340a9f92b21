"""Host logic of the serving loop, on the CPU with a fake batch and a fake
clock: request and arrival generation, the convergence rule, FIFO admission
under a device-memory budget, release on convergence, latency bookkeeping,
and the plain one-at-a-time baseline."""
import math

import numpy as np
import pytest

from paper_2312_14742_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


def decay_U(req, steps):
    """A superficial velocity that relaxes exponentially with a request-dependent time."""
    tau = 200.0 + 10.0 * req.edge
    return 1e-4 * req.porosity * (1.0 - math.exp(-steps / tau))


class FakeBatch:
    """Admits while the footprint (edge^3 bytes here) fits; a step of n costs
    n * live nodes * 1e-10 s of fake time."""

    def __init__(self, clock, budget, requests):
        self.clock = clock
        self.budget = budget
        self.used = 0
        self.by_edge_seed = {}
        self.live_boxes = {}
        self.next_slot = 0
        self.admit_order = []
        self.released_steps = {}
        self.reqs = {(r.edge, r.seed): r for r in requests}

    def admit(self, mask, periodic, g):
        req = self.reqs[(int(mask[0, 0, 0]), int(mask[0, 0, 1]))]
        need = req.edge ** 3
        if self.used + need > self.budget:
            return None
        self.used += need
        s = self.next_slot
        self.next_slot += 1
        self.live_boxes[s] = [req, 0]
        self.admit_order.append(req.id)
        return s

    def step(self, n):
        nodes = sum(b[0].edge ** 3 for b in self.live_boxes.values())
        for b in self.live_boxes.values():
            b[1] += n
        self.clock.t += n * nodes * 1e-10

    def stats(self, slots, allow_diverged=False):
        out = []
        for s in slots:
            req, steps = self.live_boxes[s]
            U = decay_U(req, steps)
            out.append({"n_fluid": req.edge ** 3, "nonfinite": 0, "max_abs_u": 3 * U, "mean_ux_superficial": U,
                        "permeability": serve.NU * U / 1e-5, "step": steps})
        return out

    def stats_queue(self, slots):
        # the fake steps synchronously: the statistics stand as of now
        self._queued = self.stats(slots, True)

    def stats_wait(self, allow_diverged=False):
        out, self._queued = self._queued, None
        return out

    def release(self, s):
        req, steps = self.live_boxes.pop(s)
        self.used -= req.edge ** 3
        self.released_steps[req.id] = steps

    @property
    def live(self):
        return len(self.live_boxes)

    def close(self):
        pass


def fake_geometry(req):
    m = np.zeros((2, 2, 2), np.uint8)
    m[0, 0, 0] = req.edge % 256
    m[0, 0, 1] = req.seed % 256
    return m


def test_make_requests_is_deterministic_and_in_range():
    a = serve.make_requests(500, 1234)
    b = serve.make_requests(500, 1234)
    assert [(r.edge, r.porosity, r.radius, r.seed) for r in a] == [(r.edge, r.porosity, r.radius, r.seed) for r in b]
    assert all(r.edge in serve.EDGES for r in a)
    assert all(0.3 <= r.porosity < 0.95 and 3.0 <= r.radius < 10.0 for r in a)
    assert [r.seed for r in a] == list(range(1234, 1734))
    # every edge value drawn, none much more often than uniform
    counts = np.bincount([serve.EDGES.index(r.edge) for r in a], minlength=len(serve.EDGES))
    assert counts.min() > 0 and counts.max() < 3 * 500 / len(serve.EDGES)


def test_poisson_arrivals():
    t = serve.poisson_arrivals(20000, 4.0, 99)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.25) < 0.01  # mean gap 1/rate
    assert abs(gaps.std() - 0.25) < 0.015  # exponential: std = mean
    assert np.all(serve.poisson_arrivals(5, 0.0, 1) == 0)


def test_convergence_rule():
    c = serve.Convergence(1e-6, 1000)
    assert c.update(1.0, 100) is None
    assert c.update(1.0 + 1e-5, 200) is None
    assert c.update(1.0 + 1e-5 + 5e-7, 300) == "converged"
    c = serve.Convergence(1e-6, 300)
    assert c.update(1.0, 100) is None and c.update(2.0, 200) is None and c.update(3.0, 300) == "cap"
    assert serve.Convergence(1e-6, 300).update(float("nan"), 100) == "diverged"
    assert serve.Convergence(1e-6, 300).update(1.0, 100, finite=False) == "diverged"
    # 16-bit storage: the tolerance sits above the stochastic-rounding noise of the mean
    c16 = serve.Convergence(1e-6, 1000, "f16s", n_fluid=10000)
    assert c16.tol == pytest.approx(8 * 2.0 ** -11 / 100)
    assert serve.Convergence(1e-6, 1000, "f16s", n_fluid=10 ** 12).tol == 1e-6
    assert serve.Convergence(1e-6, 1000, "f32", n_fluid=10).tol == 1e-6


def test_batched_server_fifo_budget_and_latency():
    reqs = serve.make_requests(40, 77, edges=(32, 48, 64, 80))
    arr = serve.poisson_arrivals(40, 50.0, 77)
    for r, a in zip(reqs, arr):
        r.arrival = float(a)
    clock = FakeClock()
    budget = 3 * 80 ** 3
    fb = FakeBatch(clock, budget, reqs)
    srv = serve.BatchedServer(storage="f32", chunk=100, tol=1e-6, cap=20000, batch=fb, clock=clock,
                              sleep=clock.sleep)
    res = srv.run(reqs, geometry_fn=fake_geometry, workers=0)
    assert sorted(r.id for r in res) == list(range(40))
    # admitted strictly in arrival order
    assert fb.admit_order == [r.id for r in sorted(reqs, key=lambda r: r.arrival)]
    assert fb.used == 0 and fb.live == 0
    for r in res:
        req = reqs[r.id]
        assert r.status == "converged"
        assert r.steps % 100 == 0
        # the first check where the change over 100 steps fell below tol
        U = lambda s: decay_U(req, s)  # noqa: E731
        s = r.steps
        assert abs(U(s) - U(s - 100)) < 1e-6 * U(s)
        assert s == 200 or abs(U(s - 100) - U(s - 200)) >= 1e-6 * U(s - 100)
        assert r.admitted >= r.arrival and r.finished > r.admitted
        assert r.latency == pytest.approx(r.finished - r.arrival)
        assert r.permeability == pytest.approx(serve.NU * U(s) / 1e-5)
    summ = serve.summarize(res, srv.fluid_updates)
    assert summ["requests"] == 40 and summ["status"]["converged"] == 40
    assert summ["p99_latency_s"] >= summ["p50_latency_s"] > 0


def test_overlap_gives_the_serial_answers():
    """The overlapped server admits while a chunk runs and takes the chunk's
    statistics afterwards: every request gets the same steps, status and
    permeability as with the serial server, and no box is stepped past the
    chunk that answered it."""
    reqs = serve.make_requests(25, 55, edges=(32, 48, 64))
    arr = serve.poisson_arrivals(25, 40.0, 55)
    for r, a in zip(reqs, arr):
        r.arrival = float(a)
    out = {}
    for overlap in (False, True):
        clock = FakeClock()
        fb = FakeBatch(clock, 4 * 64 ** 3, reqs)
        srv = serve.BatchedServer(batch=fb, clock=clock, sleep=clock.sleep, overlap=overlap)
        res = {r.id: r for r in srv.run(reqs, geometry_fn=fake_geometry, workers=0)}
        assert len(res) == 25 and fb.live == 0 and fb.used == 0
        assert fb.admit_order == [r.id for r in sorted(reqs, key=lambda r: (r.arrival, r.id))]
        for i, r in res.items():
            assert fb.released_steps[i] == r.steps
        out[overlap] = (res, srv.fluid_updates)
    ser, ovl = out[False][0], out[True][0]
    for i in ser:
        assert (ser[i].steps, ser[i].status, ser[i].permeability) == (ovl[i].steps, ovl[i].status, ovl[i].permeability)
    assert out[True][1] == out[False][1] == sum(r.n_fluid * r.steps for r in ser.values())


def test_request_larger_than_the_budget_is_an_error():
    reqs = serve.make_requests(1, 5, edges=(64,))
    clock = FakeClock()
    fb = FakeBatch(clock, 10, reqs)
    srv = serve.BatchedServer(batch=fb, clock=clock, sleep=clock.sleep)
    with pytest.raises(RuntimeError):
        srv.run(reqs, geometry_fn=fake_geometry, workers=0)


class FakeBox:
    def __init__(self, clock, reqs, edge):
        self.clock = clock
        self.reqs = reqs
        self.edge = edge
        self.steps = 0
        self.req = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass

    def set_geometry(self, mask):
        self.req = self.reqs[(int(mask[0, 0, 0]), int(mask[0, 0, 1]))]

    def step(self, n):
        self.steps += n
        self.clock.t += n * self.edge ** 3 * 1e-10

    def reduce(self, allow_diverged=False):
        U = decay_U(self.req, self.steps)
        return {"n_fluid": self.edge ** 3, "nonfinite": 0, "max_abs_u": 3 * U, "mean_ux_superficial": U,
                "permeability": serve.NU * U / 1e-5}


def test_plain_server_is_first_come_first_served():
    reqs = serve.make_requests(12, 31, edges=(32, 64))
    for i, r in enumerate(reqs):
        r.arrival = 0.01 * i
    clock = FakeClock()
    table = {(r.edge, r.seed): r for r in reqs}
    res, updates = serve.serve_plain(reqs, geometry_fn=fake_geometry, clock=clock, sleep=clock.sleep, workers=0,
                                     make_box=lambda e: FakeBox(clock, table, e))
    assert [r.id for r in res] == list(range(12))
    for a, b in zip(res, res[1:]):
        assert b.admitted >= a.finished  # one at a time
    assert updates == sum(r.n_fluid * r.steps for r in res)
    assert serve.permeability_diff(res, res) == 0.0


def test_a_diverged_request_is_released_and_the_rest_converge():
    reqs = serve.make_requests(6, 91, edges=(32, 48))
    clock = FakeClock()
    fb = FakeBatch(clock, 10 ** 9, reqs)
    poisoned = reqs[2]
    real_stats = fb.stats

    def stats(slots, allow_diverged=False):
        out = real_stats(slots, allow_diverged)
        for s, st in zip(slots, out):
            if fb.live_boxes[s][0] is poisoned:
                st["nonfinite"] = 7
        return out
    fb.stats = stats
    srv = serve.BatchedServer(batch=fb, clock=clock, sleep=clock.sleep)
    res = {r.id: r for r in srv.run(reqs, geometry_fn=fake_geometry, workers=0)}
    assert res[poisoned.id].status == "diverged" and res[poisoned.id].steps == 100
    assert all(r.status == "converged" for i, r in res.items() if i != poisoned.id)
    assert fb.live == 0


def test_live_work_cap():
    """With a cap on live nodes, no more than the cap is ever live (except a
    single box larger than it), and every request is still served in order."""
    reqs = serve.make_requests(30, 17, edges=(32, 64, 96))
    for r in reqs:
        r.arrival = 0.0
    clock = FakeClock()
    fb = FakeBatch(clock, 10 ** 12, reqs)
    peak = [0]
    real_step = fb.step

    def step(n):
        peak[0] = max(peak[0], sum(b[0].edge ** 3 for b in fb.live_boxes.values()))
        real_step(n)
    fb.step = step
    cap = 2 * 96 ** 3
    srv = serve.BatchedServer(batch=fb, clock=clock, sleep=clock.sleep, max_live_nodes=cap)
    res = srv.run(reqs, geometry_fn=fake_geometry, workers=0)
    assert len(res) == 30 and peak[0] <= cap
    assert fb.admit_order == list(range(30))


def test_batch_bench_serving_mix_respects_the_cap():
    """The batched-throughput tool's serving mix follows the request stream
    in order, skipping requests that would exceed the live-node cap."""
    from paper_2312_14742_gb300 import batch_bench

    cap = 2 * 64 ** 3
    masks = batch_bench.serving_mix(20236222, cap_nodes=cap, max_boxes=6)
    assert 0 < len(masks) <= 6
    assert sum(m.size for m in masks) <= cap
    edges = [m.shape[0] for m in masks]
    expected, tot = [], 0
    for r in serve.make_requests(400, 20236222):
        if tot + r.edge ** 3 > cap:
            continue
        expected.append(r.edge)
        tot += r.edge ** 3
        if len(expected) == 6:
            break
    assert edges == expected
    assert all(m.dtype == np.uint8 and m.shape == (e, e, e) for m, e in zip(masks, edges))
