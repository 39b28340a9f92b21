"""The C ABI from plain C: a client compiled with gcc against
include/lbm_tau1.h and linked to the library steps a channel through the
entry points alone, and gets what the Python binding gets."""
import os
import subprocess

import numpy as np
import pytest

import lbm_inputs
from paper_2312_14742_gb300 import Tau1, build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <stdlib.h>
#include "lbm_tau1.h"

int main(void)
{
    lbm_tau1_config cfg = {0};
    cfg.q = LBM_D3Q19;
    cfg.storage = LBM_F64;
    cfg.layout = LBM_DENSE;
    cfg.scheme = LBM_SCHEME_TAU1;
    cfg.nx = 8; cfg.ny = 6; cfg.nz = 20;
    cfg.periodic[0] = 1; cfg.periodic[1] = 1; cfg.periodic[2] = 0;
    cfg.kernel = LBM_KERNEL_AUTO;
    cfg.g[0] = 1e-6;
    lbm_tau1* h = NULL;
    if (lbm_tau1_create(&cfg, &h) != LBM_OK) { fprintf(stderr, "%s\n", lbm_tau1_last_error(NULL)); return 1; }
    const int n = cfg.nx * cfg.ny * cfg.nz;
    unsigned char* solid = (unsigned char*)calloc(n, 1);
    for (int i = 0; i < cfg.nx * cfg.ny; ++i) { solid[i] = 1; solid[n - 1 - i] = 1; }
    if (lbm_tau1_set_geometry(h, solid, 0) != LBM_OK) return 2;
    if (lbm_tau1_step(h, 500) != LBM_OK) return 3;
    lbm_tau1_stats st;
    if (lbm_tau1_reduce(h, &st) != LBM_OK) { fprintf(stderr, "%s\n", lbm_tau1_last_error(h)); return 4; }
    double* ux = (double*)malloc(sizeof(double) * n);
    if (lbm_tau1_get_fields(h, NULL, ux, NULL, NULL, 0) != LBM_OK) return 5;
    printf("%lld %.17g %.17g", (long long)st.step, st.mean_ux_superficial, ux[cfg.nx * cfg.ny * 10]);
    lbm_tau1_destroy(h);
    free(solid);
    free(ux);
    return 0;
}
"""


def test_c_client_matches_the_binding(tmp_path):
    build.build()
    src = tmp_path / "client.c"
    src.write_text(C_SRC)
    exe = tmp_path / "client"
    libdir = os.path.dirname(build.LIB)
    subprocess.run(["gcc", "-std=c11", "-O1", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-l:" + os.path.basename(build.LIB), "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    step, mean_ux, ux_mid = r.stdout.split()
    solid = lbm_inputs.channel(8, 6, 20)
    with Tau1(19, (8, 6, 20), storage="f64", periodic=(1, 1, 0), g=(1e-6, 0, 0)) as t:
        t.set_geometry(solid)
        t.step(500)
        s = t.reduce()
        ux = t.get_fields()[1]
    assert int(step) == 500
    assert float(mean_ux) == s["mean_ux_superficial"]
    assert float(ux_mid) == ux[10, 0, 0]
