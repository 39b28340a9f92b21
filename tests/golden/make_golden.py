"""Writes the stored expected values of tests/golden from the FP64 oracle.

Run: python tests/golden/make_golden.py (needs gcc; calls only oracle/ and
the seeded input generators). The channel case is the 32^3 Poiseuille
workload (walls z = 0 and 31, periodic x and y, g_x = 1e-6, rho = 1, u = 0 at
t = 0) at t = 1000; every (x, y) column is the same, so one column is stored.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import lbm_inputs  # noqa: E402
import oracle  # noqa: E402

G = 1e-6
STEPS = 1000


def channel_column(q: int):
    solid = lbm_inputs.channel(32, 32, 32)
    D = oracle.Domain(q, solid, periodic=(1, 1, 0), g=(G, 0.0, 0.0))
    out = D.tau1_run(D.zero_state(), STEPS)
    return {"drho": [float(v) for v in out[0][:, 0, 0]], "ux": [float(v) for v in out[1][:, 0, 0]]}


def main():
    data = {
        "source": "FP64 oracle (oracle/tau1_oracle.c), written by tests/golden/make_golden.py",
        "case": "32^3 channel, walls z=0 and z=31, periodic x and y, g_x=1e-6, rho=1 u=0 at t=0, 1000 Tau1 steps",
        "g": G, "steps": STEPS,
        "D3Q19": channel_column(19),
        "D3Q27": channel_column(27),
    }
    with open(os.path.join(HERE, "channel_t1000.json"), "w") as f:
        json.dump(data, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
