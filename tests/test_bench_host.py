"""Host logic of bench.py on the CPU: the max over ranks of a replica run
(two gloo ranks), the reference arm's rank behaviour under torchrun, and the
byte accounting."""
import importlib.util
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_module():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = bench_module()
    got = b.max_over_ranks(1.5 + rank, dist, torch.device("cpu"))
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 2.5, 1: 2.5}


def test_max_over_ranks_single_process():
    b = bench_module()
    assert b.max_over_ranks(3.25, None, None) == 3.25


def test_reference_arm_on_a_nonzero_rank_does_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.parametrize("storage,b", (("f64", 64), ("f32", 32), ("f16s", 16), ("bf16s", 16)))
def test_bytes_per_fluid_node(storage, b):
    assert bench_module().bytes_per_fluid_node(storage) == b


def test_paper_baseline_only_for_the_papers_exact_workload():
    """vs_baseline divides by the paper's figure only where Table
    tab:perf_comp has one for the same lattice, size, layout and precision
    (D2Q9 on a 4000^2 plane, FP32 1981 and FP64 1020 MFLUPS); the default
    256^3 porous D3Q19 workload has none."""
    import types

    b = bench_module()

    def a(**kw):
        base = dict(q=19, size=256, layout="dense", storage="f32")
        base.update(kw)
        return types.SimpleNamespace(**base)

    assert b.paper_baseline(a()) is None
    assert b.paper_baseline(a(q=9, size=4000))["value"] == 1.981
    assert b.paper_baseline(a(q=9, size=4000, storage="f64"))["value"] == 1.020
    assert b.paper_baseline(a(q=9, size=4000, storage="f16s")) is None
    assert b.paper_baseline(a(q=9, size=2000)) is None
    assert b.paper_baseline(a(q=9, size=4000, layout="sparse")) is None
