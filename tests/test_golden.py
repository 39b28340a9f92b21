"""Stored expected values (tests/golden): the paper's Table tab_complexity,
and the oracle's 32^3 channel at t = 1000 written by make_golden.py.

The table pins the byte accounting of the benchmark and of batch admission;
the channel file pins the oracle against an accidental change of its
arithmetic (it is also checked here against the independent 1D recurrence
of the channel)."""
import importlib.util
import json
import os

import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import build, lbm

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
GOLD = os.path.join(HERE, "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def bench_module():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_table_complexity_is_consistent():
    t = load("tab_complexity.json")
    for lat, q, d in (("D2Q9", 9, 2), ("D3Q19", 19, 3), ("D3Q27", 27, 3)):
        assert t["lbm"][lat]["AB"] == 2 * q and t["lbm"][lat]["traffic"] == 2 * q
        assert t["tau1"][lat]["traffic"] == 2 * (d + 1)
        assert t["tau1"][lat]["traffic_reduction"] == t["lbm"][lat]["traffic"] / t["tau1"][lat]["traffic"]


@pytest.mark.parametrize("storage,s", (("f64", 8), ("f32", 4), ("f16s", 2), ("bf16s", 2)))
def test_bench_bytes_match_the_table(storage, s):
    t = load("tab_complexity.json")
    b = bench_module()
    assert b.bytes_per_fluid_node(storage) == t["tau1"]["D3Q19"]["traffic"] * s
    assert b.bytes_per_fluid_node(storage, 27) == t["tau1"]["D3Q27"]["traffic"] * s
    assert b.bytes_per_fluid_node(storage, 9) == t["tau1"]["D2Q9"]["traffic"] * s


@pytest.mark.parametrize("storage,s", (("f64", 8), ("f32", 4), ("f16s", 2), ("bf16s", 2)))
def test_batch_footprint_is_the_table_memory_plus_flags(storage, s):
    build.build()
    lbm.load()
    t = load("tab_complexity.json")
    n = 64 ** 3
    fp = lbm.lbm_tau1_batch_footprint(lbm.STORAGE[storage], 64, 64, 64)
    assert fp == t["tau1"]["D3Q19"]["memory"] * s * n + n  # 256-byte multiples already


@pytest.mark.parametrize("q", (19, 27))
def test_oracle_reproduces_stored_channel(q):
    gold = load("channel_t1000.json")
    solid = lbm_inputs.channel(3, 2, 32)
    D = oracle.Domain(q, solid, periodic=(1, 1, 0), g=(gold["g"], 0, 0))
    out = D.tau1_run(D.zero_state(), gold["steps"])
    assert np.array_equal(out[1][:, 1, 2], np.array(gold[f"D3Q{q}"]["ux"]))
    assert np.array_equal(out[0][:, 1, 2], np.array(gold[f"D3Q{q}"]["drho"]))


@pytest.mark.parametrize("q", (19, 27))
def test_stored_channel_is_the_1d_recurrence(q):
    """Channel: rho stays 1 and u(z) follows u' = 2/3 v + 1/6 (v(z-1) + v(z+1)),
    v = u + g, with halfway bounce-back rows at the walls."""
    gold = load("channel_t1000.json")
    g = gold["g"]
    u = np.zeros(32)
    for _ in range(gold["steps"]):
        v = u + g
        new = np.zeros(32)
        for z in range(1, 31):
            if z == 1:
                new[z] = 0.5 * v[1] + v[2] / 6.0
            elif z == 30:
                new[z] = 0.5 * v[30] + v[29] / 6.0
            else:
                new[z] = 2.0 / 3.0 * v[z] + (v[z - 1] + v[z + 1]) / 6.0
        u = new
    ux = np.array(gold[f"D3Q{q}"]["ux"])
    assert np.max(np.abs(ux - u)) <= 1e-12 * np.max(np.abs(u))
