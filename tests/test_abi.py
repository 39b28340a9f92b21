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
    assert ctypes.sizeof(lbm.lbm_tau1_batch_config) == 40


STRUCTS = {
    "lbm_tau1_config": lbm.lbm_tau1_config,
    "lbm_tau1_stats": lbm.lbm_tau1_stats,
    "lbm_tau1_batch_config": lbm.lbm_tau1_batch_config,
}


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof and every offsetof of the header's structs, printed by a C
    program compiled against include/lbm_tau1.h, equal the binding's."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm_tau1.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(ln.split()[0], ln.split()[1]): int(ln.split()[2]) for ln in out if ln.strip()}
    for name, cls in STRUCTS.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_batch_footprint_and_cpu_errors(lib):
    lbm.load()
    # two 16-byte-record copies and one flag byte per node, each rounded up to 256 bytes
    assert lbm.lbm_tau1_batch_footprint(lbm.LBM_F32, 32, 32, 32) == 2 * 32 ** 3 * 16 + 32 ** 3
    assert lbm.lbm_tau1_batch_footprint(lbm.LBM_F16S, 3, 5, 7) == 2 * 1024 + 256  # 105 nodes * 8 B = 840 B
    assert lbm.lbm_tau1_batch_footprint(lbm.LBM_F64, 10, 10, 10) == 2 * 32000 + 1024
    assert lbm.lbm_tau1_batch_footprint(9, 4, 4, 4) == 0
    assert lbm.lbm_tau1_batch_footprint(lbm.LBM_F32, 0, 4, 4) == 0
    cfg = lbm.lbm_tau1_batch_config()
    cfg.q, cfg.storage, cfg.capacity = 19, lbm.LBM_F32, 0
    st, b = lbm.lbm_tau1_batch_create(cfg)
    assert st == lbm.LBM_EINVAL and b is None
    assert "capacity" in lbm.lbm_tau1_last_error(None)
    cfg.capacity, cfg.variant = 4, 7
    st, b = lbm.lbm_tau1_batch_create(cfg)
    assert st == lbm.LBM_EINVAL and "variant" in lbm.lbm_tau1_last_error(None)
    assert lbm.lbm_tau1_batch_step(None, 1) == lbm.LBM_EINVAL
    assert lbm.lbm_tau1_batch_destroy(None) == lbm.LBM_OK
    assert lbm.lbm_tau1_batch_live(None) == 0


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
    # the sparse layout is for the Tau1 scheme; layouts other than dense and sparse are rejected
    cfg.q, cfg.storage, cfg.layout, cfg.scheme = 19, lbm.LBM_F32, lbm.LBM_SPARSE, lbm.LBM_SCHEME_BGK
    st, h = lbm.lbm_tau1_create(cfg)
    assert st == lbm.LBM_EINVAL and "sparse" in lbm.lbm_tau1_last_error(None)
    cfg.layout, cfg.scheme = 5, lbm.LBM_SCHEME_TAU1
    st, h = lbm.lbm_tau1_create(cfg)
    assert st == lbm.LBM_EINVAL and "layout" in lbm.lbm_tau1_last_error(None)
