"""The C ABI library loads without a GPU and exports every entry point that
include/*.h declares; the Python binding declares the same set. No compute
call is made here."""
import ctypes
import glob
import os
import re

import pytest

from paper_2312_14742_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("lbm_tau1_create", "lbm_tau1_set_geometry", "lbm_tau1_step", "lbm_tau1_reduce",
                     "lbm_tau1_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(lbm.SIGNATURES) == declared_functions()


def test_struct_layouts():
    # lbm_tau1_config: 7 int32, 4 uint8, 3 doubles, one pointer
    assert ctypes.sizeof(lbm.lbm_tau1_config) == 64
    assert lbm.lbm_tau1_config.g.offset == 32
    assert ctypes.sizeof(lbm.lbm_tau1_stats) == 4 * 8 + 8 * 8


def test_abi_version_and_cpu_errors(lib):
    lbm.load()
    assert lbm.lbm_tau1_abi_version() == 1
    cfg = lbm.lbm_tau1_config()
    cfg.q = 21
    cfg.nx = cfg.ny = cfg.nz = 4
    st, h = lbm.lbm_tau1_create(cfg)
    assert st == lbm.LBM_EINVAL and h is None
    assert "q must be" in lbm.lbm_tau1_last_error(None)
    assert lbm.lbm_tau1_step(None, 1) == lbm.LBM_EINVAL
    assert lbm.lbm_tau1_destroy(None) == lbm.LBM_OK
