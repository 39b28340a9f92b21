#!/usr/bin/env python3
"""Benchmark of the Tau1 hot path (GFLUPS and fraction of the HBM roofline).

Default workload: D3Q19 Tau1, FP32 storage, dense layout, 256^3 periodic box
with overlapping solid spheres of radius 8 added from a seed until porosity
<= 0.9, body force g_x = 1e-5 (the paper's porous-media setting, Section 4.3,
at GPU scale). One step = one Tau1 update of the whole box, i.e. one launch
of the step kernel. GFLUPS = fluid nodes x steps / seconds / 1e9 (the paper's
FLUPS, Section 4).

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_inputs  # noqa: E402

WORKLOAD_INDEX = 1  # seed family of the 256^3 porous workload
SERVE_INDEX = 5     # seed family of the serving requests
METRIC = "D3Q19 Tau1 GFLUPS & % HBM roofline; serve p50/p99 latency vs plain"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=2000)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--q", type=int, default=19, choices=[9, 19, 27],
                   help="lattice; 9 (D2Q9) steps a size x size channel, the paper's 2D case")
    p.add_argument("--layout", default="dense", choices=["dense", "sparse", "compact"])
    p.add_argument("--storage", default="f32")
    p.add_argument("--kernel", default="auto")
    p.add_argument("--variant", type=int, default=-1,
                   help="tile variant of the step kernel (profiling a fixed kernel); -1: autotune")
    p.add_argument("--size", type=int, default=256)
    p.add_argument("--porosity", type=float, default=0.9)
    p.add_argument("--radius", type=float, default=8.0)
    p.add_argument("--gx", type=float, default=1e-5)
    p.add_argument("--reps", type=int, default=5, help="timed repetitions of K steps; median reported")
    p.add_argument("--cpu-steps", type=int, default=3, help="oracle steps of the full box for cpu_baseline")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-reps", type=int, default=3, help="end-to-end repetitions (median)")
    p.add_argument("--no-bgk", action="store_true", help="skip the stored-population BGK comparator")
    p.add_argument("--no-serve", action="store_true", help="skip the serving comparison")
    p.add_argument("--serve-requests", type=int, default=60)
    p.add_argument("--serve-max-edge", type=int, default=128)
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region (NVML read-only queries through ctypes)
# ---------------------------------------------------------------------------

REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, index: int, period_s: float = 0.01):
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        self.period = period_s
        self._stop = threading.Event()
        self._t = None
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            self.dev = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.dev)) != 0:
                raise OSError("no NVML handle")
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self._reason_fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(self.nvml, "nvmlDeviceGetCurrentClocksThrottleReasons")
        except (OSError, AttributeError):
            self.nvml = None

    def _run(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk)) == 0:
                self.samples.append(clk.value)
            if self._reason_fn(self.dev, ctypes.byref(rs)) == 0:
                self.reasons |= rs.value
            time.sleep(self.period)

    def __enter__(self):
        if self.nvml is not None:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._t:
            self._t.join()

    def summary(self):
        if self.nvml is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvml unavailable"]}
        names = [n for b, n in REASONS.items() if self.reasons & b and n != "gpu_idle"]
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                "sm_max_mhz": self.max_mhz, "reasons": names, "samples": len(self.samples)}


# ---------------------------------------------------------------------------

def workload(args):
    n = args.size
    if args.q == 9:
        # the paper's 2D geometry (Section 3.3, Section 4): a channel, solid rows y = 0 and n - 1
        solid = np.zeros((1, n, n), np.uint8)
        solid[0, 0] = 1
        solid[0, n - 1] = 1
        info = argparse.Namespace(porosity=float(np.mean(solid == 0)), spheres=0)
        return solid, info
    seed = lbm_inputs.workload_seed(WORKLOAD_INDEX, 0)
    solid, info = lbm_inputs.sphere_pack(n, n, n, args.radius, args.porosity, seed)
    return solid, info


def workload_name(args, info):
    if args.q == 9:
        return (f"D2Q9 Tau1 {args.storage} {args.layout}, {args.size} x {args.size} channel (solid rows y = 0 and "
                f"{args.size - 1}), periodic, g_x={args.gx:g}")
    return (f"D3Q{args.q} Tau1 {args.storage} {args.layout}, {args.size}^3 periodic, overlapping spheres "
            f"r={args.radius:g} to porosity {args.porosity:g} (reached {info.porosity:.4f}, {info.spheres} spheres), "
            f"g_x={args.gx:g}")


def bytes_per_fluid_node(storage: str, q: int = 19) -> int:
    # 2 (d+1) s: one read and one write of (rho, u) per fluid node (Section 2.1.3)
    s = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}[storage]
    d = 2 if q == 9 else 3
    return 2 * (d + 1) * s


# The paper's own figures for exactly a workload this bench can run (Table
# tab:perf_comp): D2Q9 Tau1 on a dense 4000^2 plane, best thread count, on a
# Core i9-12900K (68 GB/s measured). CPU numbers: context for vs_baseline,
# not a target. The bench's plane adds two solid rows (0.05 % of the nodes).
PAPER_FIGURES = {(9, 4000, "dense", "f32"): 1.981, (9, 4000, "dense", "f64"): 1.020}


def paper_baseline(args):
    """(GFLUPS, source) of the paper's figure for this exact workload, or None."""
    v = PAPER_FIGURES.get((args.q, args.size, args.layout, args.storage))
    if v is None:
        return None
    return {"value": v, "unit": "GFLUPS", "hardware": "Core i9-12900K (CPU, 68 GB/s measured)",
            "source": "Table tab:perf_comp, D2Q9 on 4000^2"}


TILED_KERNEL_SOURCES = ("tau1_tiled.cu", "tau1_tiled_tma.cu", "tau1_rowpair.cu", "rowpair.cuh", "tile_column.cuh",
                        "tma.cuh", "tau1_node.cuh", "pack2.cuh", "common.cuh", "lattice.cuh", "static_for.cuh",
                        "kernels.h")


def kernel_source_hash() -> str:
    """Hash of the sources the tiled step kernel is built from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2312_14742_gb300", "csrc")
    for f in TILED_KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(args):
    """DRAM bytes per launch from the committed ncu summary of this workload,
    if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", f"tau1_d3q{args.q}_{args.storage}_{args.size}_traffic.json")
    if args.layout != "dense" or args.q == 9 or not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(args, solid, nsteps):
    import oracle
    D = oracle.Domain(args.q, solid, periodic=(1, 1, 1), g=(args.gx, 0, 0))
    st = D.zero_state()
    nf = int(np.count_nonzero(solid == 0))
    st = D.tau1_step(st)  # warm-up
    t0 = time.perf_counter()
    for _ in range(nsteps):
        st = D.tau1_step(st)
    dt = time.perf_counter() - t0
    nz = solid.shape[0]
    box = f"{args.size} x {args.size} plane" if args.q == 9 else f"{args.size}^3 box"
    # the oracle's threads share the z planes: a plane (nz = 1) runs on one
    return {"value": nf * nsteps / dt / 1e9, "unit": "GFLUPS", "cores": min(oracle.get_threads(), nz),
            "kind": "oracle", "sample": f"{nsteps} FP64 oracle steps of the full {box}, OpenMP over z"}


# ---------------------------------------------------------------------------

def run_reference(args):
    """The FP64 CPU oracle on the same workload. Each step is one full oracle
    step (OpenMP over z) of a bounded sample: the whole box when the run fits
    about a minute of host time, else a slab of contiguous z planes of the
    box (periodic in z, so each node's update costs what it costs in the
    box), sized from a calibration step of a thin slab."""
    import oracle
    solid, info = workload(args)
    nz = solid.shape[0]
    g = (args.gx, 0, 0)

    def slab(planes: int):
        z0 = (nz - planes) // 2
        sub = np.ascontiguousarray(solid[z0:z0 + planes])
        return oracle.Domain(args.q, sub, periodic=(1, 1, 1), g=g), int(np.count_nonzero(sub == 0))

    Dc, nfc = slab(min(nz, 8))
    st = Dc.tau1_step(Dc.zero_state())
    t0 = time.perf_counter()
    Dc.tau1_step(st)
    rate = nfc / max(time.perf_counter() - t0, 1e-6)  # fluid nodes per second
    budget = 60.0  # seconds of host time for warm-up and timed steps together
    per_step = rate * budget / max(1, args.warmup + args.steps)
    planes = int(min(nz, max(2, per_step * nz // max(1, int(np.count_nonzero(solid == 0))))))
    D, nf = slab(planes)
    st = D.zero_state()
    for _ in range(args.warmup):
        st = D.tau1_step(st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = D.tau1_step(st)
    dt = time.perf_counter() - t0
    v = nf * args.steps / dt / 1e9
    what = "the whole box" if planes == nz else f"a slab of {planes} contiguous z planes of the box (periodic in z)"
    desc = f"{what}, {nf} fluid nodes per step, one full FP64 oracle step each, OpenMP over z"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GFLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, info)},
            "cpu_baseline": {"value": v, "unit": "GFLUPS", "cores": min(oracle.get_threads(), planes),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "GFLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2312_14742_gb300 import Tau1, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()

    solid, info = workload(args)
    nz, ny, nx = solid.shape
    n = solid.size
    nf = int(np.count_nonzero(solid == 0))
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    t = Tau1(args.q, (nx, ny, nz), storage=args.storage, periodic=(1, 1, 1), g=(args.gx, 0, 0),
             kernel=args.kernel, stream=stream, layout=args.layout)
    t.set_geometry(solid)
    t.step(min(args.warmup, 50))
    if args.variant >= 0:
        t.set_variant(args.variant)
        variant, tuned_ms = args.variant, None
    else:
        variant, tuned_ms = t.autotune(20)
    t.step(args.warmup)
    barrier()

    # device-timed region: K steps, inputs resident in HBM (working set > L2)
    times = []
    launches0 = t.launch_count
    with ClockSampler(local) as clocks:
        for _ in range(max(1, args.reps)):
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t.step(args.steps)
            e1.record(stream)
            barrier()
            times.append(e0.elapsed_time(e1) / 1e3)
    launches = (t.launch_count - launches0) // max(1, args.reps)
    dt = max_over_ranks(statistics.median(times), dist, dev)
    stats = t.reduce(allow_diverged=True)

    # end-to-end through the C ABI with host buffers: geometry in, K steps, fields out
    e2e = None
    if not args.no_e2e:
        pin_mask = torch.from_numpy(solid.reshape(-1)).pin_memory()
        outs = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(4)]
        from paper_2312_14742_gb300 import lbm as L
        e2e_times, st = [], 0
        for _ in range(args.e2e_reps):
            barrier()
            h0 = time.perf_counter()
            st |= L.lbm_tau1_set_geometry(t.h, pin_mask.data_ptr(), 0)
            st |= L.lbm_tau1_step(t.h, args.steps)
            st |= L.lbm_tau1_get_fields(t.h, *[o.data_ptr() for o in outs], 0)
            barrier()
            e2e_times.append(time.perf_counter() - h0)
        e2e_dt = max_over_ranks(statistics.median(e2e_times), dist, dev)
        if st == 0:
            e2e = {"value": world * nf * args.steps / e2e_dt / 1e9, "unit": "GFLUPS",
                   "h2d_bytes_per_step": n / args.steps, "d2h_bytes_per_step": 4 * 8 * n / args.steps,
                   "what": "set_geometry(host mask) + K steps + get_fields(host, FP64) through the C ABI",
                   "reps": args.e2e_reps, "statistic": "median"}
    t.close()

    # comparator: standard BGK at tau = 1 with stored populations, same box
    bgk = None
    if not args.no_bgk and args.storage in ("f32", "f64") and args.q != 9 and args.layout == "dense":
        from paper_2312_14742_gb300.lbm import LBM_SCHEME_BGK
        tb = Tau1(args.q, (nx, ny, nz), storage=args.storage, periodic=(1, 1, 1), g=(args.gx, 0, 0),
                  stream=stream, scheme=LBM_SCHEME_BGK)
        tb.set_geometry(solid)
        tb.step(min(args.warmup, 50))
        kb = max(10, min(args.steps, 300))
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tb.step(kb)
        e1.record(stream)
        barrier()
        bdt = e0.elapsed_time(e1) / 1e3
        tb.close()
        s = 8 if args.storage == "f64" else 4
        # 2 q s bytes per fluid node (Table tab_complexity) + one 4-byte word of wall links per node
        bbytes = 2 * args.q * s * nf + 4 * n
        bgk_value = nf * kb / bdt / 1e9
        peak_b, kind_b = measured_peaks()
        bgk = {"scheme": "BGK tau=1, stored populations (pull, AB, SoA), wall links from a per-node bit mask",
               "value": bgk_value, "unit": "GFLUPS", "steps": kb, "ms_per_step": bdt / kb * 1e3,
               "algorithmic_bytes_per_launch": bbytes, "achieved_GBps": bbytes / (bdt / kb) / 1e9,
               "frac": bbytes / (bdt / kb) / 1e9 / peak_b, "peak_kind": f"{kind_b} hbm_gbs",
               "tau1_over_bgk": None,
               "table_traffic_ratio": args.q / 4.0,
               "table_note": "traffic per node 2 q s (BGK, AB) over 2 (d+1) s (Tau1), Table tab_complexity"}

    # serving: Poisson permeability requests, continuously batched vs one at a time (rank 0)
    serve_out = None
    if rank == 0 and not args.no_serve and args.q != 9:
        from paper_2312_14742_gb300 import serve
        edges = tuple(e for e in serve.EDGES if e <= args.serve_max_edge)
        serve_out = serve.compare(args.serve_requests, lbm_inputs.workload_seed(SERVE_INDEX, 0), edges,
                                  ("f32", "f16s"), load=0.8, calib=16)
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    algo_bytes = bytes_per_fluid_node(args.storage, args.q) * nf + n  # + 1 B mask per node
    if bgk is not None:
        bgk["tau1_over_bgk"] = (nf * args.steps / dt / 1e9) / bgk["value"]
    launch_s = dt / args.steps
    achieved = algo_bytes / launch_s / 1e9
    value = world * nf * args.steps / dt / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GFLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
        "data": "synthetic",
        "config": {"workload": workload_name(args, info), "n_nodes": n, "n_fluid": nf,
                   "l2": "inputs larger than L2 (two state copies + flags exceed 126 MB); no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU", "reps": args.reps,
                   "kernel": args.kernel, "variant": variant, "autotune_ms": tuned_ms},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "traffic": ncu_traffic(args),
                     "algorithmic_bytes_per_launch": algo_bytes},
        "clocks": clocks.summary(),
        "gpu_launches": int(launches),
        "e2e": e2e,
        "bgk_comparator": bgk,
        "stats": {"permeability": stats["permeability"], "max_abs_u": stats["max_abs_u"]},
        "serve": serve_out,
    }
    paper = paper_baseline(args)
    if paper is not None:
        line["vs_baseline"] = value / paper["value"]
        line["baseline"] = paper
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args, solid, args.cpu_steps)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
