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
          g: float = 1e-5, seed_index: int = 3, peak_gbs: float | None = None) -> list[dict]:
    import torch

    import lbm_inputs
    from .lbm import LBM_SPARSE, Tau1

    stream = torch.cuda.current_stream()
    s = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}[storage]
    out = []
    for i, phi in enumerate(phis):
        t0 = time.perf_counter()
        solid, info = lbm_inputs.sphere_pack(size, size, size, radius, phi, lbm_inputs.workload_seed(seed_index, i))
        gen_s = time.perf_counter() - t0
        n = solid.size
        nf = int(np.count_nonzero(solid == 0))
        row = {"porosity_target": phi, "porosity": info.porosity, "spheres": info.spheres, "n_nodes": n,
               "n_fluid": nf, "geometry_s": gen_s}
        for layout, name in ((0, "dense"), (LBM_SPARSE, "sparse")):
            with Tau1(q, (size, size, size), storage=storage, g=(g, 0, 0), layout=layout, stream=stream) as t:
                t.set_geometry(solid)
                if layout == 0:
                    t.autotune(10)
                dt = measure(t, steps, warmup, stream)
                st = t.reduce(allow_diverged=True)
            algo = 8 * s * nf + (n if layout == 0 else 4 * (q - 1) * nf)
            r = {"gflups": nf * steps / dt / 1e9, "ms_per_step": dt / steps * 1e3,
                 "algorithmic_bytes_per_step": algo, "achieved_GBps": algo / (dt / steps) / 1e9,
                 "permeability": st["permeability"]}
            if peak_gbs:
                r["frac_of_peak"] = r["achieved_GBps"] / peak_gbs
            row[name] = r
        out.append(row)
        print(json.dumps(row), flush=True)
    return out


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
    rows = sweep(a.size, a.radius, [float(p) for p in a.phis.split(",")], a.steps, a.warmup, a.q, a.storage,
                 peak_gbs=peak)
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"size": a.size, "radius": a.radius, "steps": a.steps, "warmup": a.warmup, "q": a.q,
                       "storage": a.storage, "peak_gbs": peak, "rows": rows}, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
