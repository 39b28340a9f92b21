"""Precision run: permeability and max |u| with 16-bit storage against FP64.

A porous box (overlapping spheres of radius r to porosity phi, periodic,
body force g_x) is run to steady state once per storage format. The
convergence rule: the relative change of the superficial mean velocity U
over 100 steps below tol. With 16-bit storage U carries stochastic-rounding
noise of about 2^-p / sqrt(N_f) relative, and the tolerance is raised to 8
times that floor where it exceeds tol (the same rule as the serving loop).
After convergence the permeability and max |u| are averaged over `window`
further checks. FP64 storage is the reference; its GPU path is checked
against the FP64 oracle at small sizes by the test suite.

Usage: python -m paper_2312_14742_gb300.precision_run [--size 512] [--porosity 0.5] [--radius 12]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def run_one(solid, storage: str, g: float, tol: float, cap: int, window: int, q: int = 19) -> dict:
    from .lbm import Tau1
    from .serve import Convergence

    nz, ny, nx = solid.shape
    t0 = time.perf_counter()
    with Tau1(q, (nx, ny, nz), storage=storage, g=(g, 0, 0)) as t:
        t.set_geometry(solid)
        t.autotune(5)
        conv = None
        steps = 0
        status = None
        while status is None:
            t.step(100)
            steps += 100
            s = t.reduce(allow_diverged=True)
            if conv is None:
                conv = Convergence(tol, cap, storage, s["n_fluid"])
            status = conv.update(s["mean_ux_superficial"], steps, s["nonfinite"] == 0 and s["max_abs_u"] <= 0.3)
        ks, us = [s["permeability"]], [s["max_abs_u"]]
        for _ in range(window):
            t.step(100)
            s = t.reduce(allow_diverged=True)
            ks.append(s["permeability"])
            us.append(s["max_abs_u"])
    return {"storage": storage, "status": status, "steps": steps, "tol": conv.tol, "n_fluid": s["n_fluid"],
            "permeability": float(np.mean(ks)), "permeability_spread": float(np.std(ks)),
            "max_abs_u": float(np.mean(us)), "max_abs_u_spread": float(np.std(us)), "seconds": time.perf_counter() - t0}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--porosity", type=float, default=0.5)
    ap.add_argument("--radius", type=float, default=12.0)
    ap.add_argument("--gx", type=float, default=1e-5)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--cap", type=int, default=30000)
    ap.add_argument("--window", type=int, default=10)
    ap.add_argument("--storages", default="f64,f32,f16s,bf16s")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import lbm_inputs

    from . import build

    build.build()
    solid, info = lbm_inputs.sphere_pack(a.size, a.size, a.size, a.radius, a.porosity, lbm_inputs.workload_seed(4, 0))
    res = {"size": a.size, "porosity": info.porosity, "spheres": info.spheres, "radius": a.radius, "gx": a.gx,
           "tol": a.tol, "runs": []}
    ref = None
    for st in a.storages.split(","):
        r = run_one(solid, st, a.gx, a.tol, a.cap, a.window)
        if st == "f64":
            ref = r
        if ref is not None and st != "f64":
            r["rel_err_permeability"] = abs(r["permeability"] - ref["permeability"]) / abs(ref["permeability"])
            r["rel_err_max_abs_u"] = abs(r["max_abs_u"] - ref["max_abs_u"]) / abs(ref["max_abs_u"])
        res["runs"].append(r)
        print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
