"""Porosity sweep: GFLUPS of the dense and the sparse layout against porosity.

The paper measures its porous-media kernels on boxes with a growing number of
solid spheres (Section 4.3); here overlapping spheres of radius r are added
to a box of edge n from a seed until the porosity reaches each target. For
each porosity both layouts step the same medium: the dense tiled kernel
(every node of the box) and the sparse kernel (fluid list with a neighbour
table). GFLUPS counts fluid node updates. The algorithmic bytes per step are
32 B per fluid node plus 1 B per node for the dense layout (its flag byte is
replaced by the NaN marker in the state), and 32 + 4 (q - 1) B per fluid node
for the sparse layout (the neighbour indices).

The compact layout (dense records, work split by tile column: no fluid ->
skipped, fluid fraction >= f* -> tiled kernel, else a 4-byte node list) is
timed at the tile variant and threshold its autotune picks, and with that
variant at f* = 0 (every non-empty tile column tiled: the paper's chunk
skipping, Section 3.2) and f* = 1.01 (every fluid node through the list). Its algorithmic bytes are the dense
layout's 32 B per fluid node, plus 1 B per node of the tiled columns and 4 B
per listed node.

fit() applies the paper's porous bandwidth model (Section 4.3, B_est) to the
f* = 0 runs, with tile columns as chunks: B_max is the tiled kernel's
bandwidth on a box without solid nodes, phi_chunk the porosity of the
non-empty tile columns, R_mixed the share of non-empty columns that hold a
solid node; delta_p is fitted by least squares. It also fits the list
kernel's cost per node from the f* = 1.01 runs and predicts the split
layout's time as tiled nodes / rate_tiled + listed nodes / rate_list.

Usage: python -m paper_2312_14742_gb300.porosity_sweep [--size 512] [--steps 1000] [--warmup 2000]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

PHIS = (0.2, 0.35, 0.5, 0.65, 0.8, 0.95)


def measure(t, steps: int, warmup: int, stream) -> float:
    import torch

    t.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def sweep(size: int, radius: float, phis, steps: int, warmup: int, q: int = 19, storage: str = "f32",
          g: float = 1e-5, seed_index: int = 3, peak_gbs: float | None = None) -> tuple[list[dict], dict]:
    import torch

    import lbm_inputs
    from .lbm import LBM_COMPACT, LBM_SPARSE, Tau1

    stream = torch.cuda.current_stream()
    s = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}[storage]
    dims = (size, size, size)
    # the tiled kernel on a box without solid nodes: B_max of the model
    with Tau1(q, dims, storage=storage, g=(g, 0, 0), stream=stream) as t:
        t.set_geometry(np.zeros((size, size, size), np.uint8))
        t.autotune(10)
        dt = measure(t, steps, warmup // 4, stream)
    n = size ** 3
    full = {"ms_per_step": dt / steps * 1e3, "bytes_per_node": 8 * s + 1,
            "B_max_GBps": (8 * s + 1) * n / (dt / steps) / 1e9}
    print(json.dumps({"full_fluid": full}), flush=True)
    out = []
    for i, phi in enumerate(phis):
        t0 = time.perf_counter()
        solid, info = lbm_inputs.sphere_pack(size, size, size, radius, phi, lbm_inputs.workload_seed(seed_index, i))
        gen_s = time.perf_counter() - t0
        nf = int(np.count_nonzero(solid == 0))
        row = {"porosity_target": phi, "porosity": info.porosity, "spheres": info.spheres, "n_nodes": n,
               "n_fluid": nf, "geometry_s": gen_s}
        runs = (("dense", 0, None), ("sparse", LBM_SPARSE, None), ("compact", LBM_COMPACT, "tune"),
                ("compact_tiles", LBM_COMPACT, 0.0), ("compact_list", LBM_COMPACT, 1.01))
        tuned_variant = 0
        for name, layout, thr in runs:
            with Tau1(q, dims, storage=storage, g=(g, 0, 0), layout=layout, stream=stream) as t:
                if isinstance(thr, float):
                    # the fixed-threshold runs take the tile variant the tuned run chose
                    t.set_variant(tuned_variant)
                    t.set_compact_threshold(thr)
                t.set_geometry(solid)
                if layout == 0 or thr == "tune":
                    t.autotune(10)
                k = steps if thr in (None, "tune") else max(steps // 4, 50)
                dt = measure(t, k, warmup if thr in (None, "tune") else warmup // 8, stream)
                st = t.reduce(allow_diverged=True)
                ci = t.compact_info() if layout == LBM_COMPACT else None
                if thr == "tune":
                    tuned_variant = ci["variant"]
            if layout == 0:
                algo = 8 * s * nf + n
            elif layout == LBM_SPARSE:
                algo = 8 * s * nf + 4 * (q - 1) * nf
            else:
                algo = 8 * s * nf + ci["tiled_nodes"] + 4 * ci["listed_nodes"]
            r = {"gflups": nf * k / dt / 1e9, "ms_per_step": dt / k * 1e3,
                 "algorithmic_bytes_per_step": algo, "achieved_GBps": algo / (dt / k) / 1e9,
                 "permeability": st["permeability"]}
            if ci is not None:
                r["compact"] = ci
            if peak_gbs:
                r["frac_of_peak"] = r["achieved_GBps"] / peak_gbs
            row[name] = r
        out.append(row)
        print(json.dumps(row), flush=True)
    return out, full


def fit(rows: list[dict], full: dict) -> dict:
    """The paper's B_est (Section 4.3) on the f* = 0 runs, and a two-rate model
    of the split layout (see the module docstring)."""
    bmax = full["B_max_GBps"]
    bpn = full["bytes_per_node"]
    pts = []
    for r in rows:
        c = r["compact_tiles"]["compact"]
        nonempty = c["columns"] - c["empty_columns"]
        phi_chunk = r["n_fluid"] / c["tiled_nodes"]
        r_mixed = (nonempty - c["full_columns"]) / nonempty
        # measured bandwidth for fluid nodes, counted as the model counts it
        b_fluid = bpn * r["n_fluid"] / (r["compact_tiles"]["ms_per_step"] * 1e-3) / 1e9
        pts.append((phi_chunk, r_mixed, b_fluid))
    # B = phi_chunk bmax / (1 + d R / 2)  <=>  phi_chunk bmax / B - 1 = d R / 2
    xs = np.array([p[1] / 2 for p in pts])
    ys = np.array([p[0] * bmax / p[2] - 1 for p in pts])
    delta_p = float(np.dot(xs, ys) / np.dot(xs, xs)) if np.dot(xs, xs) > 0 else 0.0
    model = []
    for (phi_chunk, r_mixed, b_fluid), r in zip(pts, rows):
        b_est = phi_chunk * bmax / (1 + delta_p * r_mixed / 2)
        model.append({"porosity": r["porosity"], "phi_chunk": phi_chunk, "R_mixed": r_mixed,
                      "B_fluid_GBps": b_fluid, "B_est_GBps": b_est, "B_phi_chunk_GBps": phi_chunk * bmax})
    # list kernel: seconds per listed node (least squares through the origin)
    ln = np.array([r["compact_list"]["compact"]["listed_nodes"] for r in rows], dtype=np.float64)
    lt = np.array([r["compact_list"]["ms_per_step"] * 1e-3 for r in rows])
    s_list = float(np.dot(ln, lt) / np.dot(ln, ln))
    s_tile = full["ms_per_step"] * 1e-3 / rows[0]["n_nodes"]
    pred = []
    for r in rows:
        c = r["compact"]["compact"]
        t = c["tiled_nodes"] * s_tile + c["listed_nodes"] * s_list
        pred.append({"porosity": r["porosity"], "threshold": c["threshold"], "predicted_ms": t * 1e3,
                     "measured_ms": r["compact"]["ms_per_step"]})
    return {"B_max_GBps": bmax, "delta_p": delta_p, "b_est": model,
            "tiled_ns_per_node": s_tile * 1e9, "list_ns_per_node": s_list * 1e9,
            "break_even_fraction": s_tile / s_list, "split_prediction": pred}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--radius", type=float, default=12.0)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=2000)
    ap.add_argument("--q", type=int, default=19)
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--phis", default=",".join(str(p) for p in PHIS))
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
    rows, full = sweep(a.size, a.radius, [float(p) for p in a.phis.split(",")], a.steps, a.warmup, a.q, a.storage,
                       peak_gbs=peak)
    model = fit(rows, full)
    print(json.dumps({"fit": model}), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"size": a.size, "radius": a.radius, "steps": a.steps, "warmup": a.warmup, "q": a.q,
                       "storage": a.storage, "peak_gbs": peak, "full_fluid": full, "rows": rows, "fit": model},
                      f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
