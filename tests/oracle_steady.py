"""FP64 oracle references for the 16-bit storage tests: the oracle run to a
steady state, or for a fixed number of steps with a window average."""
import numpy as np

import oracle


def oracle_to_steady(q, solid, per, g, tol=1e-7, check=100, cap=60000):
    """Oracle run until the superficial mean velocity changes by less than
    tol (relative) over `check` steps; returns (stats, state, steps)."""
    D = oracle.Domain(q, solid, periodic=per, g=g)
    st = D.zero_state()
    prev = None
    steps = 0
    r = None
    while steps < cap:
        st = D.tau1_run(st, check)
        steps += check
        r = D.reduce(st)
        u = r["mean_ux_superficial"]
        if prev is not None and abs(u - prev) < tol * abs(u):
            break
        prev = u
    return r, st, steps


def oracle_window(q, solid, per, g, steps, samples=10, every=50):
    """Oracle permeability averaged over `samples` states `every` steps apart
    after `steps` steps (the same window as the 16-bit runs)."""
    D = oracle.Domain(q, solid, periodic=per, g=g)
    st = D.tau1_run(D.zero_state(), steps)
    ks = []
    for _ in range(samples):
        st = D.tau1_run(st, every)
        ks.append(D.reduce(st)["permeability"])
    return float(np.mean(ks))
