"""Batched-step throughput: GFLUPS of one Batch stepping a set of boxes with
K-step CUDA graphs, on serving-like mixes and on regular sets of boxes.

Mixes: the serving loop's request stream (edges {32, ..., 256}, porosity
U(0.3, 0.95), sphere radius U(3, 10)), taken in order while the live boxes
hold at most 2^25 nodes, the serving loop's default cap. Regular sets: 8
boxes of 128^3, one box of 256^3 (the single-box benchmark's medium) and 8
ragged boxes of 96 x 80 x 72. GFLUPS counts fluid node updates; the
algorithmic bytes per step are 2 (d + 1) s bytes per fluid node plus 1 byte
per node (Table tab_complexity), against the measured HBM copy bandwidth
when MEASURED_PEAKS.json is present.

Usage: python -m paper_2312_14742_gb300.batch_bench [--storages f32,f16s] [--steps 200] [--graph 100]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

BYTES = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}


def serving_mix(seed: int, cap_nodes: int = 2 ** 25, max_boxes: int = 48):
    from .serve import geometry, make_requests

    masks, tot = [], 0
    for r in make_requests(400, seed):
        if tot + r.edge ** 3 > cap_nodes:
            continue
        masks.append(geometry(r))
        tot += r.edge ** 3
        if len(masks) >= max_boxes:
            break
    return masks


def regular_sets():
    import lbm_inputs

    return {
        "8 x 128^3": [lbm_inputs.sphere_pack(128, 128, 128, 6.0, 0.7, 100 + i)[0] for i in range(8)],
        "1 x 256^3": [lbm_inputs.sphere_pack(256, 256, 256, 8.0, 0.9, lbm_inputs.workload_seed(1, 0))[0]],
        "8 x 96x80x72": [lbm_inputs.sphere_pack(96, 80, 72, 5.0, 0.8, 300 + i)[0] for i in range(8)],
    }


def time_batch(masks, storage: str, steps: int, graph: int, reps: int = 3, variant: int = 0,
               peak_gbs: float | None = None) -> dict:
    import torch

    from .lbm import Batch

    s = torch.cuda.current_stream()
    nf = sum(int((m == 0).sum()) for m in masks)
    n = sum(int(m.size) for m in masks)
    with Batch(19, storage, capacity=max(64, len(masks)), variant=variant, graph_steps=graph) as B:
        for m in masks:
            if B.admit(m, (1, 1, 1), (1e-5, 0, 0)) is None:
                raise RuntimeError("box does not fit the batch")
        B.step(graph)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            B.step(steps)
            e1.record(s)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3 / steps)
    algo = 8 * BYTES[storage] * nf + n
    r = {"storage": storage, "boxes": len(masks), "nodes": n, "fluid_nodes": nf, "variant": variant,
         "ms_per_step": best * 1e3, "gflups": nf / best / 1e9, "achieved_GBps": algo / best / 1e9}
    if peak_gbs:
        r["frac_of_peak"] = r["achieved_GBps"] / peak_gbs
    return r


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--storages", default="f32,f16s")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--graph", type=int, default=100)
    ap.add_argument("--seeds", default="20236222,777")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    peak = None
    pk = os.path.join(root, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as f:
            peak = float(json.load(f)["hbm_gbs"])
    from . import build

    build.build()
    sets = {f"serving mix {s}": serving_mix(int(s)) for s in a.seeds.split(",")}
    sets.update(regular_sets())
    rows = []
    for name, masks in sets.items():
        for st in a.storages.split(","):
            r = time_batch(masks, st, a.steps, a.graph, peak_gbs=peak)
            r["set"] = name
            rows.append(r)
            print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"steps": a.steps, "graph": a.graph, "peak_gbs": peak, "rows": rows}, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
