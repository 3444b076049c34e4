"""The allocation-free volume-fraction entry point, called through the C ABI.

For callers that cannot allocate device memory (a host that owns all device memory through its
own pool, or a loop that must not take the device synchronisation of cudaMalloc / cudaFree):
nn4_vof_advect_residual_static keeps its scratch in a fixed device array inside the library.
This test compares it with nn4_vof_advect_residual (caller-provided workspace) on two calls in
a row with different inputs, larger grid first, bit for bit.  It lives in a file that pytest
collects last.
"""

import ctypes

import numpy as np
import pytest
import torch

from synth import column_field, sphere_ramp_field
from tests.gpu_util import need_gpu
from tests.test_gpu_flow import _velocity

pytestmark = pytest.mark.gpu


def _call_static(nn4, G, C, u, v, w, dt, compute):
    L = nn4.lib()
    fn = L.nn4_vof_advect_residual_static
    fn.restype = ctypes.c_int
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.POINTER(nn4._Grid), ctypes.POINTER(nn4._VOFParams), vp, vp, vp, vp, vp, vp, vp]
    s = torch.empty_like(C)
    Cn = torch.empty_like(C)
    g = G.c(torch.float64)
    p = nn4.vof_params(dt, compute)
    rc = fn(ctypes.byref(g), ctypes.byref(p), nn4._ptr(C), nn4._ptr(u), nn4._ptr(v), nn4._ptr(w), nn4._ptr(s),
            nn4._ptr(Cn), nn4._stream(None))
    assert rc == nn4.OK, L.nn4_last_error()
    return s, Cn


@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_static_scratch_matches_workspace_version_twice(compute):
    """Two calls in a row, the larger grid first: a scratch element the second call failed to
    write would still hold the first call's value.  Both entry points run the same kernels on
    the same inputs, so their results are compared bit for bit."""
    need_gpu()
    from paper_2401_06755_gb300 import nn4
    cm = nn4.F64 if compute == "f64" else nn4.F32
    cases = [
        ((37, 29, 41), (1 / 36,) * 3, "bubble", 2e-4, 5),
        ((33, 17, 17), (1 / 32, 1 / 64, 1 / 32), "column", 1e-4, 4),
    ]
    for n, h, kind, dt, seed in cases:
        C = column_field(n, h, 0.25, 0.25) if kind == "column" else sphere_ramp_field(n, h, (0.5, 0.4, 0.45), 0.25, 2 * h[0])
        u, v, w = _velocity(n, h, seed)
        G = nn4.Grid(n, h)
        dev = lambda a: nn4.to_field(a, G)
        Cd, ud, vd, wd = dev(C), dev(u), dev(v), dev(w)
        s_ref, Cn_ref = nn4.vof_advect_residual(G, Cd, ud, vd, wd, dt, compute=cm)
        s, Cn = _call_static(nn4, G, Cd, ud, vd, wd, dt, cm)
        torch.cuda.synchronize()
        assert torch.equal(nn4.nodes(s, G), nn4.nodes(s_ref, G)), kind
        assert torch.equal(nn4.nodes(Cn, G), nn4.nodes(Cn_ref, G)), kind


def test_static_scratch_rejects_large_grids():
    need_gpu()
    from paper_2401_06755_gb300 import nn4
    G = nn4.Grid((129, 129, 65), (1 / 128,) * 3)
    g = G.c(torch.float64)
    L = nn4.lib()
    fn = L.nn4_vof_advect_residual_static
    p = nn4.vof_params(1e-4)
    x = ctypes.c_void_p(4096)  # never dereferenced: the size check fails first
    rc = fn(ctypes.byref(g), ctypes.byref(p), x, x, x, x, ctypes.c_void_p(8192), None, None)
    assert rc == nn4.EINVAL and b"static scratch" in L.nn4_last_error()
