"""D2Q9 Tau1 kernels and constant-density (Zou-He) faces on the GPU, through
the C ABI, against the FP64 oracle and against the paper's 2D validation.

Tolerances (as in test_gpu_tau1): FP64 |drho| <= 1e-12 absolute and |u| <=
1e-12 max|u_orc|; FP32 |u| <= 1e-5 max|u_orc| (drho 1e-5 max|drho_orc| +
1e-9). The two D2Q9 kernels (one thread per node; y-marching warps with
shuffles) give the same bits.
"""
import numpy as np
import pytest

import lbm_inputs
import oracle
from paper_2312_14742_gb300 import Tau1, build

pytestmark = pytest.mark.gpu

STORAGES = ("f64", "f32", "f16s", "bf16s")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def run(q, solid, per, g, storage, nsteps, state=None, kernel="auto", pressure=None):
    nz, ny, nx = solid.shape
    with Tau1(q, (nx, ny, nz), storage=storage, periodic=per, g=g, kernel=kernel) as t:
        t.set_geometry(solid)
        if state is not None:
            t.set_fields(*state)
        if pressure is not None:
            t.set_pressure(*pressure)
        t.step(nsteps)
        return t.get_fields()


def close(out, ref, storage, tag=""):
    umax = max(float(np.max(np.abs(ref[a]))) for a in (1, 2, 3))
    dmax = float(np.max(np.abs(ref[0])))
    du = max(float(np.max(np.abs(out[a] - ref[a]))) for a in (1, 2, 3))
    dd = float(np.max(np.abs(out[0] - ref[0])))
    if storage == "f64":
        assert dd <= 1e-12, (tag, dd)
        assert du <= 1e-12 * umax, (tag, du, umax)
    else:
        assert du <= 1e-5 * umax, (tag, du, umax)
        assert dd <= 1e-5 * dmax + 1e-9, (tag, dd, dmax)


def plane(nx, ny, fraction, seed):
    return lbm_inputs.random_mask(nx, ny, 1, fraction, seed)


@pytest.mark.parametrize("kernel", ("simple", "tiled"))
@pytest.mark.parametrize("storage,steps", [("f64", 200), ("f32", 1000)])
@pytest.mark.parametrize("per", [(1, 1, 1), (0, 1, 1), (1, 0, 1)])
def test_d2q9_matches_oracle(kernel, storage, steps, per):
    """A random porous plane of 97 x 61 (three columns of tiles, a ragged last
    one), random initial state, a body force along the periodic axes (so the
    flow does not die out against walls)."""
    solid = plane(97, 61, 0.08, 901)
    st = lbm_inputs.random_fields(solid.shape, 902, 2e-3, 3e-3, solid)
    st = (st[0], st[1], st[2], np.zeros(solid.shape))
    g = (4e-5 if per[0] else 0.0, -3e-5 if per[1] else 0.0, 0.0)
    ref = oracle.Domain(9, solid, periodic=per, g=g).tau1_run(st, steps)
    out = run(9, solid, per, g, storage, steps, state=st, kernel=kernel)
    close(out, ref, storage, (kernel, storage, per))
    assert np.all(out[3] == 0)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("dims,per", [((70, 40), (1, 1, 1)), ((31, 29), (0, 1, 1)), ((2, 5), (1, 0, 1)),
                                      ((1, 1), (1, 1, 1))])
def test_d2q9_march_bitwise_equals_simple(storage, dims, per):
    nx, ny = dims
    solid = plane(nx, ny, 0.25, 903 + nx)
    st = lbm_inputs.random_fields(solid.shape, 904, 2e-3, 3e-3, solid)
    st = (st[0], st[1], st[2], np.zeros(solid.shape))
    g = (1e-5, 2e-6, 0.0)
    a = run(9, solid, per, g, storage, 30, state=st, kernel="simple")
    b = run(9, solid, per, g, storage, 30, state=st, kernel="tiled")
    for k in range(4):
        assert np.array_equal(a[k], b[k]), (storage, dims, k)


@pytest.mark.parametrize("storage", ("f32", "f16s"))
@pytest.mark.parametrize("per", [(1, 1, 1), (1, 0, 1)])
def test_d2q9_march_bitwise_equals_simple_one_wave(storage, per):
    """A plane large enough that the march kernel sizes its row chunks to fill
    one wave of resident warps (3997 x 2999: 134 tile columns, a ragged last
    column and a ragged last chunk), against the one-thread-per-node kernel."""
    nx, ny = 3997, 2999
    solid = plane(nx, ny, 0.25, 905)
    st = lbm_inputs.random_fields(solid.shape, 906, 2e-3, 3e-3, solid)
    st = (st[0], st[1], st[2], np.zeros(solid.shape))
    g = (1e-5, 2e-6 if per[1] else 0.0, 0.0)
    a = run(9, solid, per, g, storage, 12, state=st, kernel="simple")
    b = run(9, solid, per, g, storage, 12, state=st, kernel="tiled")
    for k in range(4):
        assert np.array_equal(a[k], b[k]), (storage, per, k)


def test_d2q9_channel_steady_exact_profile():
    """Body-force channel (solid rows y = 0 and 31): the exact discrete steady
    profile u = 3 g (y - 1/2)(30.5 - y) - g/4 of the oracle pins, on the GPU."""
    g = 1e-6
    solid = np.zeros((1, 32, 40), np.uint8)
    solid[0, 0] = 1
    solid[0, 31] = 1
    out = run(9, solid, (1, 0, 1), (g, 0, 0), "f64", 20000)
    y = np.arange(1, 31, dtype=np.float64)
    exact = 3 * g * (y - 0.5) * (30.5 - y) - g / 4
    for x in (0, 17, 39):
        assert np.max(np.abs(out[1][0, 1:31, x] - exact)) <= 1e-12 * np.max(exact)


@pytest.mark.parametrize("storage", ("f64", "f32"))
@pytest.mark.parametrize("case", ["d2q9-x", "d2q9-y", "d3q19-x", "d3q27-z"])
def test_pressure_faces_match_oracle(storage, case):
    """Constant-density faces (Zou-He) on a porous box driven only by the
    density difference; GPU vs oracle after a few hundred steps."""
    q, axis = {"d2q9-x": (9, 0), "d2q9-y": (9, 1), "d3q19-x": (19, 0), "d3q27-z": (27, 2)}[case]
    if q == 9:
        solid = plane(48, 36, 0.15, 905)
        per = [1, 1, 1]
    else:
        solid, _ = lbm_inputs.sphere_pack(32, 24, 20, 3.0, 0.8, 906)
        per = [1, 1, 1]
    per[axis] = 0
    steps = 300 if storage == "f64" else 1000
    bc = (axis, 1.01, 0.99)
    ref = oracle.Domain(q, solid, periodic=per, pressure=bc).tau1_run(oracle.Domain(q, solid).zero_state(), steps)
    for kernel in ("simple", "tiled"):
        out = run(q, solid, per, (0, 0, 0), storage, steps, kernel=kernel, pressure=bc)
        close(out, ref, storage, (case, storage, kernel))


def _pressure_channel(rin, rout, steps=200000):
    nx, ny = 1000, 100
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, 0] = 1
    solid[0, ny - 1] = 1
    with Tau1(9, (nx, ny, 1), storage="f64", periodic=(0, 0, 1)) as t:
        t.set_geometry(solid)
        t.set_pressure(0, rin, rout)
        t.step(steps)
        a = t.get_fields()
        t.step(1000)
        b = t.get_fields()
    # steady: the paper's criterion, |u(t) - u(t-1)| < 1e-8 at every node
    # (here as the change over 1000 steps), and a relative change below 1e-6
    change = float(np.max(np.abs(b[1] - a[1])))
    assert change / 1000 < 1e-8 and change < 1e-6 * float(np.max(np.abs(b[1])))
    # mass flux through every cross-section (the same at steady state)
    flux = np.sum((1.0 + b[0][0]) * b[1][0], axis=0)
    spread = float((flux.max() - flux.min()) / flux.mean())
    prof = b[1][0, 1:ny - 1, 500]
    rho = 1.0 + float(np.mean(b[0][0, 1:ny - 1, 500]))
    H = ny - 2
    yp = np.arange(1, ny - 1, dtype=np.float64) - 0.5
    dpdx = (rout - rin) / 3.0 / (nx - 1)
    ana = -dpdx / (2.0 * rho * oracle.NU) * yp * (H - yp)
    mape = float(np.mean(np.abs(prof - ana) / ana)) * 100.0
    shape = float(np.mean(np.abs(prof / prof.max() - ana / ana.max()) / (ana / ana.max()))) * 100.0
    return b, mape, shape, spread


def test_paper_2d_poiseuille_mape():
    """Section 3.3: a 1000 x 100 channel, halfway bounce-back walls at the top
    and bottom rows (H = 98 fluid rows between walls at half-links), rho_in =
    1.01 and rho_out = 0.99 at the inlet and outlet (Zou-He), run to steady
    state; the profile at x = 500 against Eq. (poiseuile) with the flow from
    high to low pressure, u(y) = (-dp/dx) y' (H - y') / (2 rho nu), p = rho/3,
    nu = 1/6, y' = y - 1/2. The paper reports MAPE ~ 0.084 %.

    Read as a comparison of profile shapes (each normalised by its maximum):
    0.06 % here. The absolute profile is 0.5 % below the formula: at this
    driving the centre velocity is 0.048 (Mach 0.08), rho u is constant along
    the channel while rho falls by 2 %, and the inertia term -u^2 d(rho)/dx,
    about 0.7 % of the pressure gradient, is outside the incompressible
    formula. With a ten times smaller density difference (next test) the
    absolute error falls to 0.008 %."""
    b, mape, shape, spread = _pressure_channel(1.01, 0.99)
    print(f"MAPE {mape:.4f} %, shape MAPE {shape:.4f} %, flux spread {spread:.2e}")
    assert spread <= 1e-10
    assert shape < 0.084, shape
    assert mape < 1.0, mape
    ny = b[0].shape[1]
    assert np.all(b[0][0, 1:ny - 1, 0] == np.float64(1.01) - 1.0)


def test_low_mach_pressure_channel_matches_poiseuille():
    """The same channel at rho 1.001 / 0.999 (Mach 0.008): the absolute MAPE
    against Eq. (poiseuile) is below 0.02 %. An odd-even oscillation near the
    outlet decays more slowly at this driving, so the flux is uniform to 1e-4
    (not to rounding) after the same number of steps."""
    b, mape, shape, spread = _pressure_channel(1.001, 0.999)
    print(f"MAPE {mape:.4f} %, shape MAPE {shape:.4f} %, flux spread {spread:.2e}")
    assert spread <= 1e-4
    assert mape < 0.02, mape


@pytest.mark.parametrize("storage", STORAGES)
def test_d2q9_cylinder_array_permeability(storage):
    """A square array of cylinders (one disc of radius 6 in a periodic 32^2
    cell, solid fraction 0.11) driven by g_x = 1e-5 to steady state, both
    D2Q9 kernels: permeability within 3 % of the Hasimoto / Drummond-Tahir
    closed form (the oracle's pin) and, against the oracle run to the same
    steady state, within 1e-10 (FP64), 1e-4 (FP32) or 1 % (16-bit, the mean
    over a window of 20 states 50 steps apart)."""
    import math

    from oracle_steady import oracle_to_steady
    from test_oracle_pins import sq_array_permeability

    L = 32
    y, x = np.mgrid[0:L, 0:L]
    solid = (((x - 15.5) ** 2 + (y - 15.5) ** 2) <= 36.0).astype(np.uint8)[None]
    a = math.sqrt(int(solid.sum()) / math.pi)
    g = (1e-5, 0.0, 0.0)
    ref, _, steps = oracle_to_steady(9, solid, (1, 1, 1), g, tol=1e-7)
    want = sq_array_permeability(L, a)
    for kernel in ("simple", "tiled"):
        with Tau1(9, (L, L, 1), storage=storage, periodic=(1, 1, 1), g=g, kernel=kernel) as t:
            t.set_geometry(solid)
            t.step(steps)
            if storage in ("f64", "f32"):
                k = t.reduce()["permeability"]
                tol = 1e-10 if storage == "f64" else 1e-4
            else:
                ks = []
                for _ in range(20):
                    t.step(50)
                    ks.append(t.reduce()["permeability"])
                k = float(np.mean(ks))
                tol = 1e-2
        assert abs(k - ref["permeability"]) <= tol * abs(ref["permeability"]), (storage, kernel, k, ref)
        assert abs(k / want - 1.0) < 0.03, (storage, kernel, k, want)
