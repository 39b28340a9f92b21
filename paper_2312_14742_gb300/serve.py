"""Serving loop: permeability requests on porous samples, continuously batched.

A request is a cubic porous sample (edge, porosity, sphere radius, seed) to
be driven by a body force g_x until its superficial mean velocity stops
changing; the answer is its Darcy permeability k = nu <u_x + g_x/2> / g_x
(nu = 1/6). Requests arrive over time (Poisson). The batched server keeps
every admitted sample's state on the device in one ``Batch``: it admits
waiting requests in arrival order whenever their device footprint fits the
budget, advances all live samples together in chunks of ``chunk`` steps (one
CUDA-graph replay), reads every live sample's FP64 reductions after each
chunk, and releases a sample as soon as it has converged. The plain server
is the baseline: one sample at a time, each in its own single-box handle,
first come first served.

Admission also caps the live work: past about two waves of tile columns the
GPU is saturated, and more live boxes only lengthen every box's step, so the
batched server admits a box only while the live boxes hold at most
`max_live_nodes` nodes (the first box is always admitted). Requests beyond the
cap wait in arrival order.

Convergence: after each chunk of 100 steps, |U - U_prev| < tol |U| with U
the superficial mean u_x + g_x/2, or the step cap. With 16-bit storage the
stored state carries stochastic-rounding noise, so the mean U of N_f fluid
nodes fluctuates by about 2^-p / sqrt(N_f) relative (p = 11 FP16, 8 BF16);
the tolerance is raised to 8 times that floor where it exceeds tol.

Host and device overlap (the default): the server queues a chunk and the
statistics behind it (into page-locked memory, with an event:
``Batch.stats_queue`` / ``stats_wait``), admits waiting requests while the
chunk runs (mask upload, allocation and table edit; an admitted box joins
the next chunk), then waits for the statistics and releases the converged
boxes before it queues the next chunk, so no box is stepped past its answer.
``overlap=False`` admits only after each chunk's statistics have come back.

The host logic here only schedules; every step and reduction runs in the
CUDA library. Geometry is generated ahead of arrival on worker threads (the
generator runs in C and releases the GIL), so latency measures the server.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

EDGES = tuple(range(32, 257, 16))  # 32, 48, ..., 256
NU = 1.0 / 6.0
PRECISION_BITS = {"f16s": 11, "bf16s": 8}


@dataclass
class Request:
    id: int
    edge: int
    porosity: float
    radius: float
    seed: int
    arrival: float = 0.0  # seconds after the start of the run


@dataclass
class Result:
    id: int
    edge: int
    n_fluid: int
    steps: int
    status: str  # "converged", "cap" or "diverged"
    permeability: float
    mean_ux: float
    max_abs_u: float
    arrival: float
    admitted: float
    finished: float
    latency: float = field(init=False)

    def __post_init__(self):
        self.latency = self.finished - self.arrival


def make_requests(n: int, seed: int, edges=EDGES, porosity=(0.3, 0.95), radius=(3.0, 10.0)) -> list[Request]:
    """n requests; request i has geometry seed `seed + i`, and its edge,
    porosity and radius come from three draws of a splitmix64 stream."""
    import lbm_inputs

    u = lbm_inputs.uniform01(seed ^ 0x5E27E5, 3 * n).reshape(n, 3)
    out = []
    for i in range(n):
        e = int(edges[min(int(u[i, 0] * len(edges)), len(edges) - 1)])
        phi = porosity[0] + (porosity[1] - porosity[0]) * float(u[i, 1])
        r = radius[0] + (radius[1] - radius[0]) * float(u[i, 2])
        out.append(Request(i, e, phi, r, seed + i))
    return out


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (1/s):
    cumulative sums of exponential gaps -ln(1 - u) / rate."""
    import lbm_inputs

    if rate <= 0:
        return np.zeros(n)
    u = lbm_inputs.uniform01(seed ^ 0xA221, n)
    return np.cumsum(-np.log1p(-u) / rate)


def geometry(req: Request) -> np.ndarray:
    import lbm_inputs

    mask, _ = lbm_inputs.sphere_pack(req.edge, req.edge, req.edge, req.radius, req.porosity, req.seed)
    return mask


class Convergence:
    """Relative change of U between consecutive checks below tol, or the cap."""

    def __init__(self, tol: float, cap: int, storage: str = "f32", n_fluid: int | None = None):
        self.tol = tol
        bits = PRECISION_BITS.get(storage)
        if bits is not None and n_fluid:
            self.tol = max(tol, 8.0 * 2.0 ** -bits / math.sqrt(n_fluid))
        self.cap = cap
        self.prev = None

    def update(self, U: float, steps: int, finite: bool = True) -> str | None:
        if not finite or not math.isfinite(U):
            return "diverged"
        prev, self.prev = self.prev, U
        if prev is not None and abs(U - prev) < self.tol * abs(U):
            return "converged"
        if steps >= self.cap:
            return "cap"
        return None


class _Prefetch:
    """Geometry of upcoming requests, generated on worker threads in arrival order."""

    def __init__(self, requests, geometry_fn, depth: int, workers: int):
        self.requests = requests
        self.fn = geometry_fn
        self.depth = depth
        self.pool = ThreadPoolExecutor(max_workers=workers) if workers > 0 else None
        self.fut = {}
        self.next = 0

    def _fill(self, upto: int):
        while self.next < min(len(self.requests), upto):
            r = self.requests[self.next]
            self.fut[r.id] = self.pool.submit(self.fn, r) if self.pool else None
            self.next += 1

    def get(self, k: int, req: Request) -> np.ndarray:
        self._fill(k + 1 + self.depth)
        f = self.fut.pop(req.id, None)
        return f.result() if f is not None else self.fn(req)

    def close(self):
        if self.pool:
            self.pool.shutdown(wait=False, cancel_futures=True)


class BatchedServer:
    """Continuous batching over one ``Batch`` (see the module docstring)."""

    def __init__(self, q: int = 19, storage: str = "f32", capacity: int = 256, chunk: int = 100, tol: float = 1e-6,
                 cap: int = 20000, g: float = 1e-5, hbm_budget: int = 0, variant: int = 0, batch=None,
                 clock=time.perf_counter, sleep=time.sleep, max_live_nodes: int | None = 2 ** 25,
                 overlap: bool = True):
        if batch is None:
            from .lbm import Batch

            batch = Batch(q, storage, capacity=capacity, variant=variant, graph_steps=chunk, hbm_budget=hbm_budget)
        self.batch = batch
        self.storage = storage
        self.chunk = int(chunk)
        self.tol = tol
        self.cap = int(cap)
        self.g = float(g)
        self.clock = clock
        self.sleep = sleep
        self.max_live_nodes = max_live_nodes
        self.overlap = overlap
        self.fluid_updates = 0

    def run(self, requests: list[Request], geometry_fn=geometry, prefetch: int = 8, workers: int = 4) -> list[Result]:
        if self.overlap:
            return self._run_overlapped(requests, geometry_fn, prefetch, workers)
        order = sorted(requests, key=lambda r: (r.arrival, r.id))
        pre = _Prefetch(order, geometry_fn, prefetch, workers)
        t0 = self.clock()
        nxt = 0
        queue: deque = deque()
        live: dict[int, tuple] = {}
        results: list[Result] = []
        try:
            while len(results) < len(order):
                now = self.clock() - t0
                while nxt < len(order) and order[nxt].arrival <= now:
                    queue.append((nxt, order[nxt], None))
                    nxt += 1
                live_nodes = sum(v[0].edge ** 3 for v in live.values())
                while queue:
                    k, req, mask = queue[0]
                    if live and self.max_live_nodes and live_nodes + req.edge ** 3 > self.max_live_nodes:
                        break
                    if mask is None:
                        mask = pre.get(k, req)
                        queue[0] = (k, req, mask)
                    slot = self.batch.admit(mask, (1, 1, 1), (self.g, 0.0, 0.0))
                    if slot is None:
                        if not live:
                            raise RuntimeError(f"request {req.id} (edge {req.edge}) does not fit an empty batch")
                        break
                    queue.popleft()
                    live[slot] = (req, None, self.clock() - t0, 0)
                    live_nodes += req.edge ** 3
                if not live:
                    if nxt < len(order):
                        self.sleep(max(0.0, order[nxt].arrival - (self.clock() - t0)))
                    continue
                self.batch.step(self.chunk)
                slots = list(live)
                stats = self.batch.stats(slots, allow_diverged=True)
                now = self.clock() - t0
                for slot, st in zip(slots, stats):
                    req, conv, admitted, steps = live[slot]
                    steps += self.chunk
                    if conv is None:
                        conv = Convergence(self.tol, self.cap, self.storage, st["n_fluid"])
                    finite = st["nonfinite"] == 0 and st["max_abs_u"] <= 0.3
                    status = conv.update(st["mean_ux_superficial"], steps, finite)
                    self.fluid_updates += st["n_fluid"] * self.chunk
                    if status is None:
                        live[slot] = (req, conv, admitted, steps)
                        continue
                    results.append(Result(req.id, req.edge, st["n_fluid"], steps, status, st["permeability"],
                                          st["mean_ux_superficial"], st["max_abs_u"], req.arrival, admitted, now))
                    self.batch.release(slot)
                    del live[slot]
        finally:
            pre.close()
        return results


    def _run_overlapped(self, requests, geometry_fn, prefetch, workers) -> list[Result]:
        order = sorted(requests, key=lambda r: (r.arrival, r.id))
        pre = _Prefetch(order, geometry_fn, prefetch, workers)
        t0 = self.clock()
        nxt = 0
        queue: deque = deque()
        live: dict[int, list] = {}  # slot -> [request, convergence, admitted, steps queued]
        results: list[Result] = []

        def admit_waiting():
            nonlocal nxt
            now = self.clock() - t0
            while nxt < len(order) and order[nxt].arrival <= now:
                queue.append((nxt, order[nxt], None))
                nxt += 1
            live_nodes = sum(v[0].edge ** 3 for v in live.values())
            while queue:
                k, req, mask = queue[0]
                if live and self.max_live_nodes and live_nodes + req.edge ** 3 > self.max_live_nodes:
                    break
                if mask is None:
                    mask = pre.get(k, req)
                    queue[0] = (k, req, mask)
                slot = self.batch.admit(mask, (1, 1, 1), (self.g, 0.0, 0.0))
                if slot is None:
                    if not live:
                        raise RuntimeError(f"request {req.id} (edge {req.edge}) does not fit an empty batch")
                    break
                queue.popleft()
                live[slot] = [req, None, self.clock() - t0, 0]
                live_nodes += req.edge ** 3

        try:
            while len(results) < len(order):
                if not live:
                    admit_waiting()
                    if not live:
                        if nxt < len(order):
                            self.sleep(max(0.0, order[nxt].arrival - (self.clock() - t0)))
                        continue
                # a chunk of every live box, and its statistics behind it
                self.batch.step(self.chunk)
                slots = list(live)
                for sl in slots:
                    live[sl][3] += self.chunk
                self.batch.stats_queue(slots)
                steps_at = [live[sl][3] for sl in slots]
                # while it runs: admissions (they join the next chunk)
                admit_waiting()
                stats = self.batch.stats_wait(allow_diverged=True)
                now = self.clock() - t0
                for slot, st, steps in zip(slots, stats, steps_at):
                    req, conv, admitted, _ = live[slot]
                    if conv is None:
                        conv = Convergence(self.tol, self.cap, self.storage, st["n_fluid"])
                        live[slot][1] = conv
                    finite = st["nonfinite"] == 0 and st["max_abs_u"] <= 0.3
                    status = conv.update(st["mean_ux_superficial"], steps, finite)
                    self.fluid_updates += st["n_fluid"] * self.chunk
                    if status is None:
                        continue
                    results.append(Result(req.id, req.edge, st["n_fluid"], steps, status, st["permeability"],
                                          st["mean_ux_superficial"], st["max_abs_u"], req.arrival, admitted, now))
                    self.batch.release(slot)  # before the next chunk is queued
                    del live[slot]
        finally:
            pre.close()
        return results


def serve_plain(requests: list[Request], q: int = 19, storage: str = "f32", chunk: int = 100, tol: float = 1e-6,
                cap: int = 20000, g: float = 1e-5, geometry_fn=geometry, clock=time.perf_counter, sleep=time.sleep,
                prefetch: int = 8, workers: int = 4, make_box=None):
    """One request at a time, first come first served, each in its own
    single-box handle stepped in chunks until converged. Returns
    (results, fluid node updates)."""
    if make_box is None:
        from .lbm import Tau1

        def make_box(e):
            return Tau1(q, (e, e, e), storage=storage, g=(g, 0.0, 0.0))
    order = sorted(requests, key=lambda r: (r.arrival, r.id))
    pre = _Prefetch(order, geometry_fn, prefetch, workers)
    t0 = clock()
    results = []
    updates = 0
    try:
        for k, req in enumerate(order):
            wait = req.arrival - (clock() - t0)
            if wait > 0:
                sleep(wait)
            mask = pre.get(k, req)
            admitted = clock() - t0
            with make_box(req.edge) as t:
                t.set_geometry(mask)
                conv = None
                steps = 0
                while True:
                    t.step(chunk)
                    steps += chunk
                    st = t.reduce(allow_diverged=True)
                    if conv is None:
                        conv = Convergence(tol, cap, storage, st["n_fluid"])
                    finite = st["nonfinite"] == 0 and st["max_abs_u"] <= 0.3
                    status = conv.update(st["mean_ux_superficial"], steps, finite)
                    updates += st["n_fluid"] * chunk
                    if status is not None:
                        break
            results.append(Result(req.id, req.edge, st["n_fluid"], steps, status, st["permeability"],
                                  st["mean_ux_superficial"], st["max_abs_u"], req.arrival, admitted, clock() - t0))
    finally:
        pre.close()
    return results, updates


def summarize(results: list[Result], fluid_updates: int) -> dict:
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    span = max((r.finished for r in results), default=0.0)
    return {
        "requests": len(results),
        "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(np.mean(lat)),
        "makespan_s": span,
        "requests_per_s": len(results) / span if span > 0 else 0.0,
        "gflups": fluid_updates / span / 1e9 if span > 0 else 0.0,
        "status": {s: sum(1 for r in results if r.status == s) for s in ("converged", "cap", "diverged")},
    }


def permeability_diff(a: list[Result], b: list[Result]) -> float:
    """Largest relative permeability difference over requests served by both."""
    kb = {r.id: r.permeability for r in b}
    d = [abs(r.permeability - kb[r.id]) / abs(kb[r.id]) for r in a if r.id in kb and kb[r.id] != 0]
    return max(d) if d else 0.0


def calibrate(requests: list[Request], **server_kw) -> float:
    """Batched capacity (requests/s) on the given requests, all arriving at once."""
    reqs = [Request(r.id, r.edge, r.porosity, r.radius, r.seed, 0.0) for r in requests]
    srv = BatchedServer(**server_kw)
    try:
        res = srv.run(reqs)
    finally:
        srv.batch.close()
    return len(res) / max(r.finished for r in res)


def compare(n: int, seed: int, edges=EDGES, storages=("f32", "f16s"), load: float = 0.8, calib: int = 16,
            tol: float = 1e-6, cap: int = 20000, capacity: int = 256, q: int = 19, g: float = 1e-5,
            plain: bool = True, rate: float | None = None, max_live_nodes: int | None = 2 ** 25,
            serial: bool = False) -> dict:
    """The serving comparison: Poisson arrivals at `load` times the batched
    FP32 capacity (measured on `calib` requests of the same stream; or at a
    given `rate`), served batched in each storage format and plain (one at a
    time, FP32). With ``serial`` the batched FP32 server also runs without
    host/device overlap, for comparison."""
    reqs = make_requests(n, seed, edges)
    cap_rps = None
    if rate is None:
        cap_rps = calibrate(reqs[:calib], q=q, storage="f32", capacity=capacity, tol=tol, cap=cap, g=g,
                            max_live_nodes=max_live_nodes)
        rate = load * cap_rps
    arr = poisson_arrivals(n, rate, seed)
    for r, a in zip(reqs, arr):
        r.arrival = float(a)
    out = {"requests": n, "seed": seed, "edges": [int(e) for e in edges], "calibration_requests_per_s": cap_rps,
           "arrival_rate_per_s": rate, "load": load, "chunk": 100, "tol": tol, "cap": cap,
           "max_live_nodes": max_live_nodes}
    res = {}
    for st in storages:
        srv = BatchedServer(q=q, storage=st, capacity=capacity, tol=tol, cap=cap, g=g, max_live_nodes=max_live_nodes)
        try:
            r = srv.run(reqs)
        finally:
            srv.batch.close()
        res[st] = r
        out[f"batched_{st}"] = summarize(r, srv.fluid_updates)
    if serial:
        srv = BatchedServer(q=q, storage="f32", capacity=capacity, tol=tol, cap=cap, g=g,
                            max_live_nodes=max_live_nodes, overlap=False)
        try:
            r = srv.run(reqs)
        finally:
            srv.batch.close()
        out["batched_f32_serial"] = summarize(r, srv.fluid_updates)
        out["batched_f32_serial"]["max_rel_permeability_diff_vs_batched_f32"] = permeability_diff(r, res["f32"]) \
            if "f32" in res else None
    if plain:
        rp, up = serve_plain(reqs, q=q, storage="f32", tol=tol, cap=cap, g=g)
        res["plain"] = rp
        out["plain_f32"] = summarize(rp, up)
        for st in storages:
            out[f"batched_{st}"]["max_rel_permeability_diff_vs_plain_f32"] = permeability_diff(res[st], rp)
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=20231222 + 5000)
    ap.add_argument("--max-edge", type=int, default=256)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--calib", type=int, default=32)
    ap.add_argument("--storages", default="f32,f16s")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--serial", action="store_true", help="also run the batched FP32 server without overlap")
    ap.add_argument("--rate", type=float, default=None, help="arrival rate (1/s) instead of calibrating")
    ap.add_argument("--max-live-nodes", type=int, default=2 ** 25, help="cap on live box nodes (0: none)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    edges = tuple(e for e in EDGES if e <= a.max_edge)
    res = compare(a.requests, a.seed, edges, tuple(a.storages.split(",")), a.load, a.calib, plain=not a.no_plain,
                  rate=a.rate, max_live_nodes=a.max_live_nodes or None, serial=a.serial)
    line = json.dumps(res)
    print(line)
    if a.out:
        os.makedirs(os.path.dirname(a.out) or ".", exist_ok=True)
        with open(a.out, "w") as f:
            f.write(line + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
