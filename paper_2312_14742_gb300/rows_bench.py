"""Timings of the paths beside the 3D dense step: the D2Q9 kernels, the
constant-density (Zou-He) faces, the compact layout's node-list kernel and a
z-slab split on one GPU.

- D2Q9 (Section 3.1) on the paper's large 2D geometry, a 4000 x 4000 plane
  (Section 4): a channel with solid rows y = 0 and y = ny - 1, periodic in x,
  body force g_x = 1e-6. Both kernels (one thread per node; y-marching warps)
  and every storage format. Algorithmic bytes per fluid node: 2 (d + 1) s
  (Table tab_complexity: 24 B in FP32); the records hold four values, so the
  kernels move 2 x 4 s per node.
- Constant-density faces (Section 3.3's rho_in / rho_out) on x: the step plus
  the face kernel, against the same box stepped with periodic x and a body
  force. D2Q9 on the 4000^2 channel; D3Q19 on the 256^3 porous bench box.
- compact layout (Section 4.3's porous media, Section 5's indirect
  addressing) on a 256^3 medium of porosity 0.2: the node-list kernel alone
  (f* = 1.01) and the autotuned split.
- z-slab (one halo plane exchanged per step, Section 2.1.2's independence of
  the nodes within a step): the 256^3 bench box as two slabs on one GPU,
  exchanged through the C ABI (lbm_tau1_copy_plane) before every step, against
  the whole box. The slabs run one after the other on one device: the number
  says what the exchange and the halo planes cost, not how two GPUs scale.

CUDA events on the launching stream, after warm-up. Prints one JSON object
per line.

Usage: python -m paper_2312_14742_gb300.rows_bench [--steps 200] [--rows d2q9,faces,slab,compact] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def _time(fn, steps: int, warmup: int, stream) -> float:
    """Seconds per step of fn(k) (k steps), CUDA events on stream."""
    import torch

    fn(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / steps


def d2q9_rows(n: int, steps: int, warmup: int, stream, peak: float) -> list[dict]:
    from .lbm import Tau1

    solid = np.zeros((1, n, n), np.uint8)
    solid[0, 0] = 1
    solid[0, n - 1] = 1
    nf = int(np.count_nonzero(solid == 0))
    out = []
    for storage, s in (("f32", 4), ("f64", 8), ("f16s", 2), ("bf16s", 2)):
        for kernel in ("tiled", "simple"):
            with Tau1(9, (n, n, 1), storage=storage, periodic=(1, 0, 1), g=(1e-6, 0, 0), kernel=kernel,
                      stream=stream) as t:
                t.set_geometry(solid)
                dt = _time(t.step, steps, warmup, stream)
            algo = 6 * s * nf
            out.append({"row": "d2q9", "size": [n, n], "storage": storage,
                        "kernel": "march" if kernel == "tiled" else "simple", "ms_per_step": dt * 1e3,
                        "gflups": nf / dt / 1e9, "algorithmic_bytes_per_step": algo,
                        "achieved_GBps": algo / dt / 1e9, "frac_of_peak": algo / dt / 1e9 / peak,
                        "moved_GBps": 8 * s * nf / dt / 1e9})
    return out


def face_rows(n2: int, n3: int, steps: int, warmup: int, stream) -> list[dict]:
    import lbm_inputs
    from .lbm import Tau1

    out = []
    plane = np.zeros((1, n2, n2), np.uint8)
    plane[0, 0] = 1
    plane[0, n2 - 1] = 1
    box, _ = lbm_inputs.sphere_pack(n3, n3, n3, 8.0, 0.9, lbm_inputs.workload_seed(1, 0))
    for q, solid, dims in ((9, plane, (n2, n2, 1)), (19, box, (n3, n3, n3))):
        per_px = (1, 0, 1) if q == 9 else (1, 1, 1)
        per_face = (0, 0, 1) if q == 9 else (0, 1, 1)
        with Tau1(q, dims, storage="f32", periodic=per_px, g=(1e-6, 0, 0), stream=stream) as t:
            t.set_geometry(solid)
            base = _time(t.step, steps, warmup, stream)
        with Tau1(q, dims, storage="f32", periodic=per_face, stream=stream) as t:
            t.set_geometry(solid)
            t.set_pressure(0, 1.01, 0.99)
            faces = _time(t.step, steps, warmup, stream)
        out.append({"row": "zou_he", "q": q, "size": list(dims), "ms_per_step_periodic": base * 1e3,
                    "ms_per_step_faces": faces * 1e3, "overhead": faces / base - 1.0,
                    "face_nodes_per_step": 2 * (dims[1] * dims[2])})
    return out


def slab_rows(n: int, steps: int, warmup: int, stream) -> list[dict]:
    import lbm_inputs
    from .lbm import Tau1
    from .slab import GpuSlab, bounds, run_in_process

    solid, _ = lbm_inputs.sphere_pack(n, n, n, 8.0, 0.9, lbm_inputs.workload_seed(1, 0))
    with Tau1(19, (n, n, n), storage="f32", g=(1e-5, 0, 0), stream=stream) as t:
        t.set_geometry(solid)
        whole = _time(t.step, steps, warmup, stream)
    slabs = []
    try:
        for r in range(2):
            z0, z1 = bounds(n, 2, r)
            s = GpuSlab(19, (n, n, n), z0, z1, storage="f32", g=(1e-5, 0, 0), stream=stream)
            s.set_geometry(solid)
            slabs.append(s)
        split = _time(lambda k: run_in_process(slabs, k), steps, warmup, stream)
    finally:
        for s in slabs:
            s.close()
    return [{"row": "z_slab", "size": [n, n, n], "slabs": 2, "ms_per_step_whole": whole * 1e3,
             "ms_per_step_two_slabs_one_gpu": split * 1e3, "overhead": split / whole - 1.0,
             "exchange_bytes_per_step": 2 * 2 * n * n * 16}]


def compact_rows(n: int, steps: int, warmup: int, stream, peak: float) -> list[dict]:
    """The compact layout on a low-porosity medium (256^3 by default, spheres
    of radius 12 to porosity 0.2, the sweep's first medium at a smaller size):
    every fluid node through the node list (f* = 1.01: the list kernel alone),
    then the autotuned split."""
    import lbm_inputs
    from .lbm import LBM_COMPACT, Tau1

    solid, _ = lbm_inputs.sphere_pack(n, n, n, 12.0, 0.2, lbm_inputs.workload_seed(3, 0))
    nf = int(np.count_nonzero(solid == 0))
    out = []
    for name in ("list", "tuned"):
        with Tau1(19, (n, n, n), storage="f32", g=(1e-5, 0, 0), layout=LBM_COMPACT, stream=stream) as t:
            if name == "list":
                t.set_compact_threshold(1.01)
            t.set_geometry(solid)
            if name == "tuned":
                t.autotune(10)
            dt = _time(t.step, steps, warmup, stream)
            ci = t.compact_info()
        algo = 32 * nf + ci["tiled_nodes"] + 4 * ci["listed_nodes"]
        out.append({"row": "compact", "split": name, "size": [n, n, n], "porosity": 1.0 - float(solid.mean()),
                    "n_fluid": nf, "ms_per_step": dt * 1e3, "gflups": nf / dt / 1e9,
                    "algorithmic_bytes_per_step": algo, "achieved_GBps": algo / dt / 1e9,
                    "frac_of_peak": algo / dt / 1e9 / peak, "compact": ci})
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--n2", type=int, default=4000, help="edge of the D2Q9 plane")
    ap.add_argument("--n3", type=int, default=256, help="edge of the 3D box")
    ap.add_argument("--rows", default="d2q9,faces,slab,compact", help="which rows to time")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    which = set(a.rows.split(","))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch

    from . import build

    build.build()
    pk = os.path.join(root, "MEASURED_PEAKS.json")
    peak, kind = (float(json.load(open(pk))["hbm_gbs"]), "measured") if os.path.exists(pk) else (6800.0, "fallback")
    stream = torch.cuda.current_stream()
    rows = []
    todo = []
    if "compact" in which:
        todo += compact_rows(a.n3, a.steps, a.warmup, stream, peak)
    if "d2q9" in which:
        todo += d2q9_rows(a.n2, a.steps, a.warmup, stream, peak)
    if "faces" in which:
        todo += face_rows(a.n2, a.n3, a.steps, a.warmup, stream)
    if "slab" in which:
        todo += slab_rows(a.n3, a.steps, a.warmup, stream)
    for r in todo:
        r["peak_GBps"] = peak
        r["peak_kind"] = kind
        rows.append(r)
        print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
