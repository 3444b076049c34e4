"""CPU checks of the C ABI: the library builds, loads, exports every declared symbol, and
rejects bad arguments on the host before any launch (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nn4.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nn4_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def nn4():
    from paper_2401_06755_gb300 import build
    build.build()
    from paper_2401_06755_gb300 import nn4 as m
    m.lib()
    return m


def test_every_declared_symbol_is_exported(nn4):
    names = _declared()
    assert len(names) >= 14
    L = nn4.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_plan_options_layout_and_shapes(nn4):
    """The binding's option struct matches the header (the trailing fields get the C defaults)."""
    o = nn4._PlanOpts()
    o.coarse_entry_nodes = 123
    o.pass_shape = 7
    nn4.lib().nn4_plan_opts_default(ctypes.byref(o))
    assert o.coarse_entry_nodes == 0 and o.pass_shape == -1 and o.autotune == 1 and o.fused_prolong == 0
    assert nn4.pass_shapes() == 5


def test_row_pitch(nn4):
    assert nn4.row_pitch(257, nn4.F64) == 272
    assert nn4.row_pitch(257, nn4.F32) == 288
    assert nn4.row_pitch(257, nn4.BF16) == 320
    assert nn4.row_pitch(33, nn4.F64) == 48
    assert nn4.lib().nn4_row_pitch(0, nn4.F64) == -1


def test_host_validation_rejects_bad_arguments(nn4):
    L = nn4.lib()
    G = nn4.Grid((9, 9, 9), (0.125,) * 3)
    g = G.c(nn4.F64)
    p = ctypes.c_void_p(4096)  # never dereferenced: validation fails first
    null = ctypes.c_void_p(0)
    assert L.nn4_stencil_apply(ctypes.byref(g), nn4.F64, null, null, p, null) == nn4.EINVAL
    assert b"NULL" in L.nn4_last_error()
    bad = G.c(nn4.F64)
    bad.pitch = 5
    assert L.nn4_stencil_apply(ctypes.byref(bad), nn4.F64, p, null, ctypes.c_void_p(8192), null) == nn4.EINVAL
    bad = G.c(nn4.F64)
    bad.h[1] = -1.0
    assert L.nn4_residual(ctypes.byref(bad), nn4.F64, p, p, null, p, null, null) == nn4.EINVAL
    even = nn4.Grid((8, 9, 9), (0.125,) * 3).c(nn4.F64)
    assert L.nn4_restrict(ctypes.byref(even), nn4.F64, p, ctypes.c_void_p(8192), null) == nn4.EINVAL
    assert L.nn4_residual_restrict(ctypes.byref(even), nn4.F64, p, p, null, ctypes.c_void_p(8192), null,
                                   null) == nn4.EINVAL
    assert L.nn4_residual_restrict(ctypes.byref(g), nn4.F64, p, p, null, p, null, null) == nn4.EINVAL  # alias
    # misaligned pointer
    assert L.nn4_stencil_apply(ctypes.byref(g), nn4.F64, ctypes.c_void_p(4100), null,
                               ctypes.c_void_p(8192), null) == nn4.EINVAL
    assert L.nn4_jacobi_smooth(ctypes.byref(g), nn4.F64, p, null, ctypes.c_void_p(8192),
                               ctypes.c_void_p(16384), ctypes.c_double(2.5), null) == nn4.EINVAL
    # plan options are validated before any allocation
    o = nn4._PlanOpts()
    L.nn4_plan_opts_default(ctypes.byref(o))
    assert o.inner == nn4.F64 and o.inner_cycles == 1 and abs(o.omega - 2 / 3) < 1e-15
    o.inner_cycles = 0
    h = ctypes.c_void_p(0)
    assert L.nn4_plan_create(ctypes.byref(g), null, ctypes.byref(o), ctypes.byref(h)) == nn4.EINVAL
    small = nn4.Grid((2, 9, 9), (0.125,) * 3).c(nn4.F64)
    L.nn4_plan_opts_default(ctypes.byref(o))
    assert L.nn4_plan_create(ctypes.byref(small), null, ctypes.byref(o), ctypes.byref(h)) == nn4.EINVAL


def test_product_path_does_not_import_the_oracle():
    """The binding and the CUDA sources never reference the oracle package."""
    pkg = os.path.join(ROOT, "paper_2401_06755_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, flags=re.M), f
                assert "oracle/" not in text, f


def test_no_unresolved_internal_symbols(nn4):
    """Every internal (nn4 namespace) symbol the library references is defined in it."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if not nm:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--undefined-only", nn4.LIB_PATH], capture_output=True, text=True).stdout
    bad = [l for l in out.splitlines() if "_ZN3nn4" in l]
    assert not bad, bad
