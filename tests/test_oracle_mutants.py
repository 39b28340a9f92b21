"""Plants plausible mistakes in a copy of the oracle and checks that the pins
catch every one of them (the oracle source itself is never modified).

Each mutant is the oracle's C source with one textual change, compiled into a
temporary directory. A compact battery of the pins of test_oracle_pins.py is
run against it; at least one pin must fail.
"""
import math
import os

import numpy as np
import pytest

import lbm_inputs
import oracle
from test_oracle_pins import brute_force_push, channel_recurrence, sc_array_permeability

SRC = os.path.join(os.path.dirname(oracle.__file__), "tau1_oracle.c")

MUTANTS = {
    "quadratic coefficient": ("4.5 * cu * cu", "4.0 * cu * cu"),
    "sign of u.u term": ("- 1.5 * vv", "+ 1.5 * vv"),
    "dropped linear term": ("3.0 * cu + ", ""),
    "bounce-back direction": ("feq_dev(L, L->inv[k], drho[i]", "feq_dev(L, k, drho[i]"),
    "bounce-back ignores force": ("ux[i] + g[0], uy[i] + g[1], uz[i] + g[2]);\n    } else",
                                  "ux[i], uy[i], uz[i]);\n    } else"),
    "push instead of pull": ("int p[3] = {x - L->c[k][0], y - L->c[k][1], z - L->c[k][2]};",
                             "int p[3] = {x + L->c[k][0], y + L->c[k][1], z + L->c[k][2]};"),
    "no division by rho": ("double r = 1.0 / (1.0 + d_acc);", "double r = 1.0;"),
    "momentum sign": ("jx += (double)L->c[k][0] * f;", "jx -= (double)L->c[k][0] * f;"),
    "edge weight": ("W19[4] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0", "W19[4] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 35.0"),
    "D3Q27 corner weight": ("1.0 / 54.0, 1.0 / 216.0}", "1.0 / 54.0, 1.0 / 200.0}"),
    "D2Q9 diagonal weight": ("W9[4] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0", "W9[4] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 32.0"),
    "Zou-He factor of the outgoing sum": ("- h0 - 2.0 * hout", "- h0 - 1.0 * hout"),
    "Zou-He face sign": ("if (pos[a] == 0) { sgn = 1.0;", "if (pos[a] == 0) { sgn = -1.0;"),
    "transposed index": ("(size_t)x + (size_t)G->nx * ((size_t)y + (size_t)G->ny * (size_t)z)",
                         "(size_t)y + (size_t)G->ny * ((size_t)x + (size_t)G->nx * (size_t)z)"),
    "wall counted as fluid": ("if (!G->periodic[a]) return 1;", "if (!G->periodic[a]) p[a] = 0;"),
    "reduction without the half-step force": ("double px = ux[i] + 0.5 * g[0]", "double px = ux[i] + 0.0 * g[0]"),
    "superficial mean over fluid nodes": ("out[2] = sx / (double)n;", "out[2] = sx / nf;"),
    "mass over all nodes": ("if (solid[i]) continue;\n        nf += 1.0;", "nf += solid[i] ? 0.0 : 1.0;"),
    "viscosity of tau = 1 in the Darcy ratio": ("(1.0 / 6.0) * out[2] / g[0]", "(1.0 / 3.0) * out[2] / g[0]"),
}


def battery(lib):
    """Returns the list of pins that fail for the given oracle library."""
    failed = []
    # lattice isotropy (second moment) and inv
    for q in (9, 19, 27):
        c, w, inv = oracle.lattice(q, lib=lib)
        cf = c.astype(float)
        want = np.eye(3) / 3
        if q == 9:
            want[2, 2] = 0.0  # one plane: no z moment
        if not np.allclose(np.einsum("k,ka,kb->ab", w, cf, cf), want, atol=1e-15):
            failed.append(f"isotropy{q}")
    # 1D channel recurrence (q = 19), 300 steps; x and y dims differ
    g = 1e-6
    D = oracle.Domain(19, lbm_inputs.channel(3, 2, 32), periodic=(1, 1, 0), g=(g, 0, 0), lib=lib)
    out = D.tau1_run(D.zero_state(), 300)
    ref = channel_recurrence(32, g, 300)
    if not np.max(np.abs(out[1][:, 0, 0] - ref)) <= 1e-12 * np.max(np.abs(ref)):
        failed.append("channel")
    # isolated node closed form
    solid = np.ones((3, 3, 3), np.uint8)
    solid[1, 1, 1] = 0
    gg = (1e-4, -2e-4, 5e-5)
    D = oracle.Domain(27, solid, g=gg, lib=lib)
    st = [np.zeros((3, 3, 3)) for _ in range(4)]
    st[0][1, 1, 1], st[1][1, 1, 1] = 0.02, 0.01
    o = D.tau1_step(st)
    exp = (0.02, -(0.01 + gg[0]), -gg[1], -gg[2])
    if any(abs(o[a][1, 1, 1] - exp[a]) > 1e-16 for a in range(4)):
        failed.append("isolated")
    # mass conservation with a non-periodic axis and random state
    solid = lbm_inputs.random_mask(6, 5, 7, 0.25, 31)
    st = lbm_inputs.random_fields(solid.shape, 32, 1e-3, 1e-3, solid)
    D = oracle.Domain(19, solid, periodic=(1, 0, 1), g=(1e-5, 0, 0), lib=lib)
    o = D.tau1_run(st, 50)
    if abs(math.fsum(o[0][solid == 0]) - math.fsum(st[0][solid == 0])) > 1e-13:
        failed.append("mass")
    # brute-force push BGK with full populations
    solid = lbm_inputs.random_mask(4, 3, 5, 0.25, 33)
    st = lbm_inputs.random_fields(solid.shape, 34, 2e-2, 3e-2, solid)
    gb = (1e-3, -2e-3, 5e-4)
    ref = brute_force_push(19, solid, (1, 0, 1), gb, st, 2)
    o = oracle.Domain(19, solid, periodic=(1, 0, 1), g=gb, lib=lib).tau1_run(st, 2)
    if any(np.max(np.abs(o[a] - ref[a])) > 1e-14 for a in range(4)):
        failed.append("brute")
    # reduction of isolated nodes after one step (closed forms: -u - g/2, sum of 1 + drho)
    solid = np.ones((4, 4, 4), np.uint8)
    solid[::2, ::2, ::2] = 0
    fl = solid == 0
    st = lbm_inputs.random_fields(solid.shape, 35, 1e-2, 2e-2, solid)
    gr = np.array([3e-5, -1e-5, 2e-5])
    D = oracle.Domain(19, solid, g=gr, lib=lib)
    r = D.reduce(D.tau1_step(st))
    phys = -st[1][fl] - 0.5 * gr[0]
    if (abs(r["mass"] - math.fsum(1.0 + st[0][fl])) > 1e-13
            or abs(r["mean_ux_superficial"] - math.fsum(phys) / solid.size) > 1e-15
            or abs(r["mean_u_fluid"][0] - math.fsum(phys) / fl.sum()) > 1e-15):
        failed.append("reduce")
    # Zou-He faces: a uniform flow between two faces of the same density is a fixed point
    solid = np.zeros((1, 3, 9), np.uint8)
    u0 = 2e-3
    st = (np.full(solid.shape, 0.01), np.full(solid.shape, u0), np.zeros(solid.shape), np.zeros(solid.shape))
    D = oracle.Domain(9, solid, periodic=(0, 1, 1), pressure=(0, 1.01, 1.01), lib=lib)
    o = D.tau1_run(st, 20)
    if np.max(np.abs(o[1] - u0)) > 1e-15 or np.max(np.abs(o[0] - 0.01)) > 1e-15:
        failed.append("zou-he uniform")
    # permeability of a simple cubic sphere array (L = 12, R = 4: the closed
    # form within 2.8 % at this resolution; 5 % allowed)
    L = 12
    zz, yy, xx = np.mgrid[0:L, 0:L, 0:L]
    solid = (((xx - 5.5) ** 2 + (yy - 5.5) ** 2 + (zz - 5.5) ** 2) <= 16.0).astype(np.uint8)
    a = (3.0 * int(solid.sum()) / (4.0 * math.pi)) ** (1.0 / 3.0)
    D = oracle.Domain(19, solid, g=(1e-6, 0.0, 0.0), lib=lib)
    k = D.reduce(D.tau1_run(D.zero_state(), 1500))["permeability"]
    if not abs(k / sc_array_permeability(L, a) - 1.0) < 0.05:
        failed.append("sphere array permeability")
    return failed


def _compile(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    out = str(tmp_path / f"lib{name}.so")
    oracle.build(force=True, src=str(src), out=out, openmp=False)
    return oracle.load(out)


def test_unmutated_oracle_passes_battery(tmp_path):
    lib = _compile(tmp_path, "clean", open(SRC).read())
    assert battery(lib) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    before, after = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(before) >= 1, f"mutation site not found: {name}"
    lib = _compile(tmp_path, "mut", text.replace(before, after, 1))
    assert battery(lib), f"no pin caught the mutant: {name}"
