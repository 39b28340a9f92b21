"""16-bit storage (FP16 and BF16 with per-field power-of-two scales, FP32
arithmetic, stochastic rounding on store): accuracy where the answer is
known, the re-scaling that keeps FP16 inside its range, and permeability
within 1% of FP64.

With stochastic rounding the stored state carries a zero-mean noise of about
one unit in the last place, so a steady state is a statistically steady one:
the 16-bit runs step as long as the FP64 run needed to converge and then
average the fields over a window."""
import numpy as np
import pytest

import lbm_inputs
from oracle_steady import oracle_to_steady
from paper_2312_14742_gb300 import Tau1, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def run_to_steady(q, solid, per, g, tol=1e-7, check=100, cap=60000):
    """FP64 run until the mean superficial velocity changes by < tol over
    `check` steps; returns (stats, fields, steps)."""
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage="f64", periodic=per, g=g) as t:
        t.set_geometry(solid)
        prev = None
        steps = 0
        while steps < cap:
            t.step(check)
            steps += check
            s = t.reduce()
            u = s["mean_ux_superficial"]
            if prev is not None and abs(u - prev) < tol * abs(u):
                break
            prev = u
        return s, t.get_fields(), steps


def run_averaged(q, solid, per, g, storage, steps, samples=20, every=50):
    """16-bit run for `steps` steps, then the mean of the fields and of the
    reduced statistics over `samples` states `every` steps apart."""
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage=storage, periodic=per, g=g) as t:
        t.set_geometry(solid)
        t.step(steps)
        acc_f = None
        acc_s = {}
        for _ in range(samples):
            t.step(every)
            s = t.reduce()
            assert s["nonfinite"] == 0
            f = t.get_fields()
            acc_f = [a.copy() for a in f] if acc_f is None else [a + b for a, b in zip(acc_f, f)]
            for k in ("permeability", "max_abs_u", "mean_ux_superficial"):
                acc_s[k] = acc_s.get(k, 0.0) + s[k]
        return {k: v / samples for k, v in acc_s.items()}, [a / samples for a in acc_f]


@pytest.mark.parametrize("storage", ("f16s", "bf16s"))
def test_uniform_acceleration_with_rescaling(storage):
    """No walls, body force: u(t) = t g exactly in real arithmetic. Over 2000
    steps u grows by 2000x from its first value, which the FP16 scale has to
    follow (checks every 64 steps). Stochastic rounding makes each store
    unbiased, so the error is a random walk of about one unit in the last
    place per step, damped by the averaging over neighbours: a few units in
    the last place of u(t)."""
    solid = np.zeros((8, 16, 32), np.uint8)
    g = (1e-6, -5e-7, 0.0)
    ulp = 2.0 ** -11 if storage == "f16s" else 2.0 ** -8
    with Tau1(19, (32, 16, 8), storage=storage, g=g) as t:
        t.set_geometry(solid)
        for n in (10, 200, 2000):
            t.step(n - t.reduce()["step"])
            d, ux, uy, _ = t.get_fields()
            # the domain mean follows t g closely (noise averages over 4096 nodes)
            assert abs(np.mean(ux) - n * g[0]) <= 2 * ulp * n * abs(g[0]), (storage, n)
            assert abs(np.mean(uy) - n * g[1]) <= 2 * ulp * n * abs(g[1]), (storage, n)
            assert np.max(np.abs(ux - n * g[0])) <= 8 * ulp * n * abs(g[0]), (storage, n)
            assert np.max(np.abs(uy - n * g[1])) <= 8 * ulp * n * abs(g[1]), (storage, n)


@pytest.mark.parametrize("storage", ("f16s", "bf16s"))
def test_small_increments_do_not_stall(storage):
    """An increment far below half a unit in the last place: with
    round-to-nearest the stored velocity would never move; with stochastic
    rounding its mean advances by g per step. u = 0.01 has a last place of
    2^-14 in BF16 (S = 1) and of 2^-17 in FP16 (S = 2^18 puts it at 2621);
    g is 1/64 of that. Over n = 4096 steps the gain is 64 last places, and
    the noise of the domain mean is about sqrt(n / 6N) ~ 0.4 last places."""
    solid = np.zeros((8, 16, 32), np.uint8)
    u0 = 0.01
    g = (2.0 ** -20, 0.0, 0.0) if storage == "bf16s" else (2.0 ** -23, 0.0, 0.0)
    n = 4096
    shape = solid.shape
    with Tau1(19, (32, 16, 8), storage=storage, g=g) as t:
        t.set_geometry(solid)
        t.set_fields(np.zeros(shape), np.full(shape, u0), np.zeros(shape), np.zeros(shape))
        d, ux0, _, _ = t.get_fields()
        t.step(n)
        d, ux, _, _ = t.get_fields()
    gain = float(np.mean(ux) - np.mean(ux0))
    assert abs(gain - n * g[0]) <= 0.05 * n * g[0], (storage, gain, n * g[0])


@pytest.mark.parametrize("storage", ("f16s", "bf16s"))
def test_channel_steady_profile(storage):
    """Steady channel (walls z = 0, 31; g_x = 1e-6): the exact discrete
    profile u(z) = 3 g (z - 1/2)(30.5 - z) - g/4 within 1% of its maximum.
    The FP16 scale of drho and u_z (both near rounding level in this flow)
    must follow the headroom rule's floors without overflowing."""
    g = 1e-6
    solid = lbm_inputs.channel(4, 4, 32)
    _, _, steps = run_to_steady(19, solid, (1, 1, 0), (g, 0, 0), tol=1e-7)
    s, f = run_averaged(19, solid, (1, 1, 0), (g, 0, 0), storage, steps)
    z = np.arange(1, 31)
    exact = 3 * g * (z - 0.5) * (30.5 - z) - g / 4
    ux = f[1][1:31].mean(axis=(1, 2))
    assert np.max(np.abs(ux - exact)) <= 1e-2 * np.max(exact), (storage, steps)


@pytest.mark.parametrize("storage", ("f16s", "bf16s"))
def test_porous_permeability_within_one_percent(storage):
    """Porosity 0.5 medium (the 512^3 workload's kind at 48^3): steady-state
    permeability and max|u| with 16-bit storage against the FP64 oracle run
    to the same steady state (relative change of the mean velocity below
    1e-7 over 100 steps): permeability within 1 %, max|u| within 2 %."""
    solid, info = lbm_inputs.sphere_pack(48, 48, 48, 5.0, 0.5, lbm_inputs.workload_seed(3, 48))
    g = (1e-5, 0.0, 0.0)
    ref, fref, steps = oracle_to_steady(19, solid, (1, 1, 1), g, tol=1e-7)
    got, fgot = run_averaged(19, solid, (1, 1, 1), g, storage, steps)
    assert abs(got["permeability"] - ref["permeability"]) <= 1e-2 * abs(ref["permeability"])
    assert abs(got["max_abs_u"] - ref["max_abs_u"]) <= 2e-2 * ref["max_abs_u"]


@pytest.mark.parametrize("storage", ("f64", "f32", "f16s", "bf16s"))
def test_sphere_array_permeability_matches_closed_form(storage):
    """One sphere (nodes within 6 of the centre) in a periodic 24^3 cell: a
    simple cubic array at solid fraction 0.066. The steady permeability is
    within 3 % of the Hasimoto / Sangani-Acrivos closed form (the oracle's
    own pin, test_oracle_pins.sc_array_permeability, with the radius of a
    ball of the solid nodes' volume) and, against the oracle run to the same
    steady state, within 1e-10 (FP64), 1e-4 (FP32) or 1 % (16-bit, averaged
    over a window)."""
    import math

    from test_oracle_pins import sc_array_permeability

    L = 24
    z, y, x = np.mgrid[0:L, 0:L, 0:L]
    solid = (((x - 11.5) ** 2 + (y - 11.5) ** 2 + (z - 11.5) ** 2) <= 36.0).astype(np.uint8)
    a = (3.0 * int(solid.sum()) / (4.0 * math.pi)) ** (1.0 / 3.0)
    g = (1e-5, 0.0, 0.0)
    ref, _, steps = oracle_to_steady(19, solid, (1, 1, 1), g, tol=1e-7)
    if storage in ("f64", "f32"):
        with Tau1(19, (L, L, L), storage=storage, periodic=(1, 1, 1), g=g) as t:
            t.set_geometry(solid)
            t.step(steps)
            got = t.reduce()
        tol = 1e-10 if storage == "f64" else 1e-4
    else:
        got, _ = run_averaged(19, solid, (1, 1, 1), g, storage, steps)
        tol = 1e-2
    k = got["permeability"]
    assert abs(k - ref["permeability"]) <= tol * abs(ref["permeability"]), (storage, k, ref["permeability"])
    assert abs(k / sc_array_permeability(L, a) - 1.0) < 0.03, (storage, k, sc_array_permeability(L, a))
