"""The C-ABI library builds, loads and exports every entry point include/lbm.h
declares; struct layouts agree between C and the binding; host-side
validation rejects bad input before any device call (no GPU needed)."""
import ctypes as C
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2605_30878_gb300 import build as lbm_build
from paper_2605_30878_gb300 import lbm
from paper_2605_30878_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def L():
    lbm_build.build()
    return lbm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_function_is_exported(L):
    names = declared_functions()
    assert set(names) == set(lbm.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    assert set(names) <= exported
    for n in names:
        assert getattr(L, n) is not None


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "lbm.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_params), sizeof(lbm_ghost),'
                   ' sizeof(lbm_probe), sizeof(lbm_diag), offsetof(lbm_params, g), offsetof(lbm_diag, step));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [C.sizeof(lbm.Params), C.sizeof(lbm.Ghost), C.sizeof(lbm.Probe), C.sizeof(lbm.Diag),
                   lbm.Params.g.offset, lbm.Diag.step.offset]


def test_domain_bytes(L):
    cfg = wl.sphere_config(n=64, R=10, R0=8)
    ng = len(cfg["ghosts"][0])
    b32 = lbm.domain_bytes(cfg["params"], ng)
    p64 = dict(cfg["params"], precision=lbm.FP64)
    b64 = lbm.domain_bytes(p64, ng)
    nn = 64 ** 3
    assert b32 >= 4 * 19 * nn * 4 + (1 + 2 * 3 + 1) * nn * 4 + nn
    assert b64 > 1.9 * b32
    assert lbm.domain_bytes(dict(cfg["params"], lattice=7), ng) == 0
    assert lbm.domain_bytes(dict(cfg["params"], lattice=9), ng) == 0          # D2Q9 needs nz == 1
    assert lbm.domain_bytes(cfg["params"], -1) == 0
    # the largest grids: populations are indexed in 32 bits, Q * plane < 2^31
    big = dict(cfg["params"], nx=480, ny=480, nz=480)
    assert lbm.domain_bytes(big, 0) > 19 * 4 * 4 * 480 ** 3        # 110.6M nodes: accepted
    assert lbm.domain_bytes(dict(big, nx=512, ny=512, nz=512), 0) == 0
    assert lbm.domain_bytes(dict(cfg["params"], lattice=9, nx=16000, ny=16000, nz=1), 0) == 0      # 9 x 256M
    assert lbm.domain_bytes(dict(cfg["params"], lattice=9, nx=15000, ny=15000, nz=1), 0) > 0       # 9 x 225M


def _create_error(params, solid, ghosts):
    with pytest.raises(lbm.LbmError) as e:
        lbm.Domain(params, solid, ghosts, workspace="library", stream=0)
    return e.value


def test_validation_before_any_device_call(L):
    cfg = wl.cylinder_config()
    P, solid, (nodes, normals) = cfg["params"], cfg["solid"], cfg["ghosts"]
    e = _create_error(dict(P, W=3.0), solid, (nodes, normals))
    assert e.status == lbm.LBM_ERR_ARG and "W" in str(e)
    e = _create_error(P, solid, (nodes[1:], normals[1:]))
    assert e.status == lbm.LBM_ERR_ARG and "ghost list" in str(e)
    bad = normals.copy()
    bad[3] *= 1.01
    e = _create_error(P, solid, (nodes, bad))
    assert e.status == lbm.LBM_ERR_ARG and "unit" in str(e)
    dup = nodes.copy()
    dup[1] = dup[0]
    e = _create_error(P, solid, (dup, normals))
    assert e.status == lbm.LBM_ERR_ARG
    e = _create_error(dict(P, periodic=1), solid, (nodes, normals))        # y not periodic, fluid on y ends
    assert e.status == lbm.LBM_ERR_ARG and "periodic" in str(e)
    e = _create_error(dict(P, rho_l=0.0), solid, (nodes, normals))
    assert e.status == lbm.LBM_ERR_ARG
    e = _create_error(dict(P, M_phi=1.0), solid, (nodes, normals))          # alpha < 0
    assert e.status == lbm.LBM_ERR_ARG and "alpha" in str(e)
    assert "alpha" in lbm.last_error(None)


def test_ghost_records_have_the_lbm_ghost_layout():
    """The binding hands lbm_create_domain a numpy record array; its layout is
    that of lbm_ghost (int64 node, then three doubles)."""
    import ctypes as C
    from paper_2605_30878_gb300 import lbm
    arr, n = lbm.ghost_array([5, 7], [[1, 0, 0], [0, 0.6, 0.8]])
    assert n == 2 and arr.dtype.itemsize == C.sizeof(lbm.Ghost) == 32
    g = (lbm.Ghost * 2).from_buffer(arr)
    assert g[1].node == 7 and list(g[1].n) == [0.0, 0.6, 0.8]
    empty, n0 = lbm.ghost_array(np.zeros(0, np.int64), np.zeros((0, 3)))
    assert n0 == 0 and len(empty) == 1


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the compiled library the binding raises."""
    from paper_2605_30878_gb300 import lbm as binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", "/nonexistent/liblbm.so")
    with pytest.raises(RuntimeError, match="missing"):
        binding.load()
