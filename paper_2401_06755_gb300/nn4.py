"""Python binding of the C ABI in include/nn4.h (argument marshalling only).

Every function here forwards to ``_lib/libnn4.so``; no step of the method runs in Python.  If the
library is missing the import of a function raises: there is no fallback path.

Fields are torch tensors of shape (nz, ny, pitch) ("storage") whose first nx entries of every row
hold the nodes; :func:`field` allocates one with the library's pitch, and :func:`nodes` returns
the (nz, ny, nx) view.  PyTorch provides device memory and streams only.
"""

import ctypes
import os
from dataclasses import dataclass, field as dc_field

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnn4.so")

OK, EINVAL, ECUDA, ENOMEM, ENOCONV, ENONFINITE, ETIMEOUT, EBOUNDS, EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
F64, F32, BF16 = 0, 1, 2
DIRICHLET, NATURAL = 0, 1
OUTER_CYCLES, OUTER_FCG = 0, 1

_TORCH = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}
_CODE = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}


class NN4Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nn4 status {code}: {msg}")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_double * 3), ("bc", ctypes.c_int32 * 6),
                ("pitch", ctypes.c_int64)]


class _PlanOpts(ctypes.Structure):
    _fields_ = [("inner", ctypes.c_int), ("inner_cycles", ctypes.c_int32), ("outer", ctypes.c_int32),
                ("omega", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("profile", ctypes.c_int32), ("inner_krylov", ctypes.c_int32),
                ("coarse_tail", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("coarse_entry_nodes", ctypes.c_int32), ("fused_prolong", ctypes.c_int32),
                ("pass_shape", ctypes.c_int32)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("cycles", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_len", ctypes.c_int32),
                ("kernels", ctypes.c_int64)]


class _VOFParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("dt", "alpha_a", "eps_k", "K_plus", "K_minus", "beta", "eps_x",
                                               "K_pos", "alpha_min", "alpha_max", "detect_hi", "detect_lo")] + \
               [("p", ctypes.c_int32), ("compute", ctypes.c_int32)]


class _FlowParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("dt", "rho_l", "rho_g", "mu_l", "mu_g", "sigma_t", "g", "alpha_a",
                                               "eps_k")] + \
               [("p", ctypes.c_int32), ("momentum_iters", ctypes.c_int32), ("correction_iters", ctypes.c_int32),
                ("pressure_cycles", ctypes.c_int32), ("pressure_rtol", ctypes.c_double), ("compute", ctypes.c_int32)]


class _FlowStats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("c_min", ctypes.c_double), ("c_max", ctypes.c_double),
                ("hs_iters", ctypes.c_int32), ("nh_iters", ctypes.c_int32), ("hs_rel", ctypes.c_double),
                ("nh_rel", ctypes.c_double)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("shape", ctypes.c_int32 * 16), ("zmax", ctypes.c_int32 * 16),
                ("jacobi_us", ctypes.c_float * 16), ("items", ctypes.c_int32 * 16), ("nodes", ctypes.c_int64 * 16)]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("n", (ctypes.c_int32 * 3) * 16), ("coarsest_free", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


_lib = None


def lib():
    """Loads libnn4.so (raising if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "python -m paper_2401_06755_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        G = ctypes.POINTER(_Grid)
        sig = {
            "nn4_row_pitch": (ctypes.c_int64, [i32, ctypes.c_int]),
            "nn4_stencil_apply": (ctypes.c_int, [G, ctypes.c_int, vp, vp, vp, vp]),
            "nn4_residual": (ctypes.c_int, [G, ctypes.c_int, vp, vp, vp, vp, vp, vp]),
            "nn4_restrict": (ctypes.c_int, [G, ctypes.c_int, vp, vp, vp]),
            "nn4_residual_restrict": (ctypes.c_int, [G, ctypes.c_int, vp, vp, vp, vp, vp, vp]),
            "nn4_prolong": (ctypes.c_int, [G, ctypes.c_int, vp, vp, ctypes.c_int, vp]),
            "nn4_jacobi_smooth": (ctypes.c_int, [G, ctypes.c_int, vp, vp, vp, vp, dbl, vp]),
            "nn4_plan_opts_default": (None, [ctypes.POINTER(_PlanOpts)]),
            "nn4_plan_create": (ctypes.c_int, [G, vp, ctypes.POINTER(_PlanOpts), ctypes.POINTER(vp)]),
            "nn4_plan_destroy": (ctypes.c_int, [vp]),
            "nn4_vcycle": (ctypes.c_int, [vp, vp, vp, vp]),
            "nn4_pressure_solve": (ctypes.c_int, [vp, vp, vp, dbl, i32, ctypes.POINTER(_SolveInfo), vp]),
            "nn4_pressure_solve_host": (ctypes.c_int, [vp, vp, vp, dbl, i32, ctypes.POINTER(_SolveInfo), vp]),
            "nn4_plan_profile": (ctypes.c_int, [vp, ctypes.POINTER(_KernelTime), i32]),
            "nn4_plan_query": (ctypes.c_int, [vp, ctypes.POINTER(_PlanInfo)]),
            "nn4_vof_params_default": (None, [ctypes.POINTER(_VOFParams), dbl]),
            "nn4_vof_workspace_bytes": (ctypes.c_int64, [G]),
            "nn4_vof_advect_residual": (ctypes.c_int, [G, ctypes.POINTER(_VOFParams), vp, vp, vp, vp, vp, vp, vp, vp]),
            "nn4_mass_sum": (ctypes.c_int, [G, vp, vp, vp]),
            "nn4_batch_create": (ctypes.c_int, [G, i32, ctypes.POINTER(_PlanOpts), ctypes.POINTER(vp)]),
            "nn4_batch_destroy": (ctypes.c_int, [vp]),
            "nn4_batch_query": (ctypes.c_int, [vp, ctypes.POINTER(_BatchInfo)]),
            "nn4_pressure_solve_batched": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dbl, i32,
                                                          ctypes.POINTER(_SolveInfo), ctypes.POINTER(ctypes.c_float),
                                                          vp]),
            "nn4_vof_advect_residual_static": (ctypes.c_int, [G, ctypes.POINTER(_VOFParams), vp, vp, vp, vp, vp, vp, vp]),
            "nn4_flow_params_default": (None, [ctypes.POINTER(_FlowParams), dbl]),
            "nn4_momentum_sources": (ctypes.c_int, [G, ctypes.POINTER(_FlowParams), vp, vp, vp, vp, vp, vp, vp]),
            "nn4_pressure_rhs_hs": (ctypes.c_int, [G, vp, vp, vp, vp, vp]),
            "nn4_pressure_rhs_hs_ex": (ctypes.c_int, [G, i32, vp, vp, vp, vp, vp]),
            "nn4_momentum_workspace_bytes": (ctypes.c_int64, [G]),
            "nn4_pressure_rhs_nh": (ctypes.c_int, [G, ctypes.POINTER(_FlowParams), vp, vp, vp, vp, vp, vp, vp]),
            "nn4_velocity_correct": (ctypes.c_int, [G, ctypes.POINTER(_FlowParams), vp, vp, vp, vp, vp, vp, vp]),
            "nn4_momentum_predict": (ctypes.c_int, [G, ctypes.POINTER(_FlowParams), vp, ctypes.POINTER(vp),
                                                    ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp,
                                                    ctypes.POINTER(vp), vp, vp]),
            "nn4_flow_create": (ctypes.c_int, [G, G, ctypes.POINTER(_FlowParams), ctypes.POINTER(_PlanOpts),
                                               ctypes.POINTER(vp)]),
            "nn4_flow_destroy": (ctypes.c_int, [vp]),
            "nn4_flow_step": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(_FlowStats), vp]),
            "nn4_last_error": (ctypes.c_char_p, []),
            "nn4_device_error": (ctypes.c_int, []),
            "nn4_version": (ctypes.c_char_p, []),
            "nn4_pass_shapes": (ctypes.c_int32, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != OK:
        raise NN4Error(code, lib().nn4_last_error().decode())
    return code


@dataclass
class Grid:
    """Vertex grid: n = (nx, ny, nz) nodes, spacing h, one of DIRICHLET / NATURAL per face."""
    n: tuple
    h: tuple
    bc: tuple = dc_field(default_factory=lambda: (NATURAL,) * 6)

    def pitch(self, dtype):
        return row_pitch(self.n[0], dtype)

    def c(self, dtype):
        g = _Grid()
        g.n[:] = list(self.n)
        g.h[:] = [float(v) for v in self.h]
        g.bc[:] = list(self.bc)
        g.pitch = self.pitch(dtype)
        return g

    def coarse(self):
        return Grid(tuple((m + 1) // 2 for m in self.n), tuple(2.0 * v for v in self.h), self.bc)


def row_pitch(nx, dtype):
    code = dtype if isinstance(dtype, int) else _CODE[dtype]
    return int(lib().nn4_row_pitch(int(nx), code))


def field(grid, dtype=torch.float64, device="cuda", fill=0.0):
    """A zero (or ``fill``) pitched storage tensor (nz, ny, pitch) for ``grid``."""
    nx, ny, nz = grid.n
    return torch.full((nz, ny, row_pitch(nx, dtype)), fill, dtype=dtype, device=device)


def nodes(storage, grid):
    """The (nz, ny, nx) view of the node values of a storage tensor."""
    return storage[:, :, :grid.n[0]]


def to_field(a, grid, dtype=torch.float64, device="cuda"):
    """Copies an (nz, ny, nx) array into a new pitched storage tensor."""
    f = field(grid, dtype, device)
    nodes(f, grid).copy_(torch.as_tensor(a).to(dtype))
    return f


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dt(t):
    return _CODE[t.dtype]


def stencil_apply(grid, x, k=None, y=None, stream=None):
    y = torch.empty_like(x) if y is None else y
    g = grid.c(x.dtype)
    _check(lib().nn4_stencil_apply(ctypes.byref(g), _dt(x), _ptr(x), _ptr(k), _ptr(y), _stream(stream)))
    return y


def residual(grid, b, x, k=None, r=None, norm2=None, stream=None):
    r = torch.empty_like(x) if r is None else r
    g = grid.c(x.dtype)
    _check(lib().nn4_residual(ctypes.byref(g), _dt(x), _ptr(b), _ptr(x), _ptr(k), _ptr(r), _ptr(norm2),
                              _stream(stream)))
    return r


def restrict(grid, r_fine, r_coarse=None, stream=None):
    if r_coarse is None:
        r_coarse = field(grid.coarse(), r_fine.dtype, r_fine.device)
    g = grid.c(r_fine.dtype)
    _check(lib().nn4_restrict(ctypes.byref(g), _dt(r_fine), _ptr(r_fine), _ptr(r_coarse), _stream(stream)))
    return r_coarse


def residual_restrict(grid, b, x, k=None, r_coarse=None, norm2=None, stream=None):
    if r_coarse is None:
        r_coarse = field(grid.coarse(), x.dtype, x.device)
    g = grid.c(x.dtype)
    _check(lib().nn4_residual_restrict(ctypes.byref(g), _dt(x), _ptr(b), _ptr(x), _ptr(k), _ptr(r_coarse),
                                       _ptr(norm2), _stream(stream)))
    return r_coarse


def prolong(grid, e_coarse, e_fine=None, accumulate=False, stream=None):
    if e_fine is None:
        e_fine = field(grid, e_coarse.dtype, e_coarse.device)
    g = grid.c(e_coarse.dtype)
    _check(lib().nn4_prolong(ctypes.byref(g), _dt(e_coarse), _ptr(e_coarse), _ptr(e_fine),
                             int(bool(accumulate)), _stream(stream)))
    return e_fine


def jacobi_smooth(grid, b, x_in, k=None, x_out=None, omega=2.0 / 3.0, stream=None):
    x_out = torch.empty_like(x_in) if x_out is None else x_out
    g = grid.c(x_in.dtype)
    _check(lib().nn4_jacobi_smooth(ctypes.byref(g), _dt(x_in), _ptr(b), _ptr(k), _ptr(x_in), _ptr(x_out),
                                   float(omega), _stream(stream)))
    return x_out


def vof_params(dt, compute=None, **over):
    """The scheme's constants with time step dt; compute: F64 (default) or F32 arithmetic."""
    p = _VOFParams()
    lib().nn4_vof_params_default(ctypes.byref(p), float(dt))
    if compute is not None:
        p.compute = int(compute)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def vof_workspace(grid, device="cuda"):
    n = lib().nn4_vof_workspace_bytes(ctypes.byref(grid.c(torch.float64)))
    return torch.empty(int(n) // 8, dtype=torch.float64, device=device)


def vof_advect_residual(grid, C, u, v, w, dt, s_C=None, C_next=None, workspace=None, params=None, stream=None,
                        compute=None):
    """One explicit volume-fraction step; returns (s_C, C_next) (FP64 storage tensors)."""
    s_C = torch.empty_like(C) if s_C is None else s_C
    C_next = torch.empty_like(C) if C_next is None else C_next
    workspace = vof_workspace(grid, C.device) if workspace is None else workspace
    p = vof_params(dt, compute) if params is None else params
    g = grid.c(torch.float64)
    _check(lib().nn4_vof_advect_residual(ctypes.byref(g), ctypes.byref(p), _ptr(C), _ptr(u), _ptr(v), _ptr(w),
                                         _ptr(s_C), _ptr(C_next), _ptr(workspace), _stream(stream)))
    return s_C, C_next


def mass_sum(grid, C, out=None, stream=None):
    out = torch.zeros(1, dtype=torch.float64, device=C.device) if out is None else out
    g = grid.c(torch.float64)
    _check(lib().nn4_mass_sum(ctypes.byref(g), _ptr(C), _ptr(out), _stream(stream)))
    return out


def device_error():
    return lib().nn4_device_error()


def version():
    return lib().nn4_version().decode()


def pass_shapes():
    """Number of compiled stencil-pass tile shapes (values of Plan(pass_shape=...))."""
    return int(lib().nn4_pass_shapes())


class Plan:
    """Multigrid hierarchy for one grid (and optional FP64 coefficient field k)."""

    def __init__(self, grid, k=None, inner=F64, inner_cycles=1, outer=OUTER_CYCLES, omega=2.0 / 3.0,
                 use_graph=True, check_every=1, profile=False, inner_krylov=0, coarse_tail=True, autotune=True,
                 coarse_entry_nodes=0, fused_prolong=False, pass_shape=-1):
        o = _PlanOpts()
        lib().nn4_plan_opts_default(ctypes.byref(o))
        o.inner, o.inner_cycles, o.outer = int(inner), int(inner_cycles), int(outer)
        o.omega, o.use_graph, o.check_every = float(omega), int(bool(use_graph)), int(check_every)
        o.profile = int(bool(profile))
        o.inner_krylov = int(inner_krylov)
        o.coarse_tail = int(bool(coarse_tail))
        o.autotune = int(bool(autotune))
        o.coarse_entry_nodes = int(coarse_entry_nodes)
        o.pass_shape = int(pass_shape)
        o.fused_prolong = int(bool(fused_prolong))
        self.grid = grid
        self.inner = inner
        self._k = k  # keep the coefficient alive while the plan exists
        self._g = grid.c(torch.float64)
        h = ctypes.c_void_p(0)
        _check(lib().nn4_plan_create(ctypes.byref(self._g), _ptr(k), ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h is not None and self._h.value:
            lib().nn4_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vcycle(self, b, x, stream=None):
        _check(lib().nn4_vcycle(self._h, _ptr(b), _ptr(x), _stream(stream)))
        return x

    def _solve(self, fn, b, x, rtol, max_iters, history_len, stream, ptr):
        hist = (ctypes.c_double * max(1, history_len))()
        info = _SolveInfo()
        info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        info.history_len = history_len
        code = fn(self._h, ptr(b), ptr(x), float(rtol), int(max_iters), ctypes.byref(info), _stream(stream))
        if code not in (OK, ENOCONV):
            _check(code)
        n = min(history_len, info.iterations + 1)
        return {"status": code, "iterations": info.iterations, "cycles": info.cycles,
                "rel_res": info.rel_res, "history": list(hist[:n]), "kernels": info.kernels}

    def profile(self):
        """{kernel category: (launches, total ms)} since the last call (profile plans only)."""
        buf = (_KernelTime * 256)()
        n = lib().nn4_plan_profile(self._h, buf, 256)
        if n < 0:
            _check(n)
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(n, 256))}

    def query(self):
        q = _PlanInfo()
        _check(lib().nn4_plan_query(self._h, ctypes.byref(q)))
        return {"levels": q.levels, "n": [tuple(q.n[l]) for l in range(q.levels)],
                "coarsest_free": q.coarsest_free, "device_bytes": q.device_bytes}

    def solve(self, b, x, rtol=1e-8, max_iters=200, history_len=512, stream=None):
        """Pressure solve on device FP64 storage tensors b, x (x: initial guess, then solution)."""
        return self._solve(lib().nn4_pressure_solve, b, x, rtol, max_iters, history_len, stream, _ptr)

    def solve_host(self, b, x, rtol=1e-8, max_iters=200, history_len=512, stream=None):
        """The same with dense (nz, ny, nx) host FP64 tensors (pinned for full copy speed)."""
        assert b.device.type == "cpu" and x.device.type == "cpu" and b.is_contiguous() and x.is_contiguous()
        return self._solve(lib().nn4_pressure_solve_host, b, x, rtol, max_iters, history_len, stream,
                           lambda t: ctypes.c_void_p(t.data_ptr()))


class Batch:
    """Many independent constant-coefficient pressure systems of uneven sizes, solved together."""

    def __init__(self, grids, inner=F32, inner_cycles=2, omega=2.0 / 3.0, check_every=1, autotune=True,
                 pass_shape=-1):
        o = _PlanOpts()
        lib().nn4_plan_opts_default(ctypes.byref(o))
        o.inner, o.inner_cycles, o.omega, o.check_every = int(inner), int(inner_cycles), float(omega), int(check_every)
        o.autotune, o.pass_shape = int(bool(autotune)), int(pass_shape)
        self.grids = list(grids)
        arr = (_Grid * len(self.grids))(*[g.c(torch.float64) for g in self.grids])
        h = ctypes.c_void_p(0)
        _check(lib().nn4_batch_create(arr, len(self.grids), ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h is not None and self._h.value:
            lib().nn4_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self):
        """The autotuner's choice per level step: shape, z cap, measured us, items, nodes."""
        info = _BatchInfo()
        _check(lib().nn4_batch_query(self._h, ctypes.byref(info)))
        return [{"level": l, "shape": info.shape[l], "zmax": info.zmax[l], "jacobi_us": info.jacobi_us[l],
                 "items": info.items[l], "nodes": info.nodes[l]} for l in range(info.levels)]

    def solve(self, bs, xs, rtol=1e-8, max_iters=100, stream=None):
        """bs, xs: lists of FP64 storage tensors.  Returns (status, infos, latency_ms)."""
        n = len(self.grids)
        bp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in bs])
        xp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs])
        infos = (_SolveInfo * n)()
        lat = (ctypes.c_float * n)()
        code = lib().nn4_pressure_solve_batched(self._h, bp, xp, float(rtol), int(max_iters), infos, lat,
                                                _stream(stream))
        if code not in (OK, ENOCONV):
            _check(code)
        return code, [{"iterations": infos[i].iterations, "rel_res": infos[i].rel_res,
                       "kernels": infos[i].kernels} for i in range(n)], list(lat)


def flow_params(dt, compute=None, **over):
    """Physical constants and scheme settings; compute: F64 (default) or F32 arithmetic of the
    explicit terms."""
    p = _FlowParams()
    lib().nn4_flow_params_default(ctypes.byref(p), float(dt))
    if compute is not None:
        p.compute = int(compute)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def _arr3(ts):
    return (ctypes.c_void_p * 3)(*[t.data_ptr() for t in ts])


def momentum_sources(grid, fp, C, stream=None):
    s = [torch.empty_like(C) for _ in range(3)]
    kappa = torch.empty_like(C)
    g = grid.c(torch.float64)
    _check(lib().nn4_momentum_sources(ctypes.byref(g), ctypes.byref(fp), _ptr(C), _ptr(s[0]), _ptr(s[1]),
                                      _ptr(s[2]), _ptr(kappa), None, _stream(stream)))
    return s, kappa


def pressure_rhs_hs(pgrid, s, stream=None, compute=F64):
    b = torch.empty_like(s[0])
    g = pgrid.c(torch.float64)
    _check(lib().nn4_pressure_rhs_hs_ex(ctypes.byref(g), int(compute), _ptr(s[0]), _ptr(s[1]), _ptr(s[2]), _ptr(b),
                                        _stream(stream)))
    return b


def pressure_rhs_nh(pgrid, fp, C, ut, stream=None):
    b = torch.empty_like(C)
    g = pgrid.c(torch.float64)
    _check(lib().nn4_pressure_rhs_nh(ctypes.byref(g), ctypes.byref(fp), _ptr(C), _ptr(ut[0]), _ptr(ut[1]),
                                     _ptr(ut[2]), _ptr(b), None, _stream(stream)))
    return b


def velocity_correct(vgrid, fp, C, dp, u, p_nh=None, stream=None):
    g = vgrid.c(torch.float64)
    _check(lib().nn4_velocity_correct(ctypes.byref(g), ctypes.byref(fp), _ptr(C), _ptr(dp), _ptr(u[0]), _ptr(u[1]),
                                      _ptr(u[2]), _ptr(p_nh), _stream(stream)))
    return u


def momentum_workspace(grid, device="cuda"):
    n = lib().nn4_momentum_workspace_bytes(ctypes.byref(grid.c(torch.float64)))
    return torch.empty(int(n) // 8, dtype=torch.float64, device=device)


def momentum_predict(vgrid, fp, C, un, uh, p, s, ut=None, uh_next=None, workspace=None, stream=None):
    """One predictor iteration from u^n (un) and u^{n+1/2} (uh); returns (u~, the next u^{n+1/2})."""
    ut = [torch.empty_like(C) for _ in range(3)] if ut is None else ut
    uh_next = [torch.empty_like(C) for _ in range(3)] if uh_next is None else uh_next
    ws = momentum_workspace(vgrid, C.device) if workspace is None else workspace
    g = vgrid.c(torch.float64)
    _check(lib().nn4_momentum_predict(ctypes.byref(g), ctypes.byref(fp), _ptr(C), _arr3(un), _arr3(uh), _arr3(ut),
                                      _arr3(uh_next), _ptr(p), _arr3(s), _ptr(ws), _stream(stream)))
    return ut, uh_next


class Flow:
    """The four-stage multiphase time step on device state (Section 2.4)."""

    def __init__(self, vgrid, pgrid, fp, inner=F64, inner_cycles=1, outer=OUTER_CYCLES, inner_krylov=0,
                 check_every=1):
        o = _PlanOpts()
        lib().nn4_plan_opts_default(ctypes.byref(o))
        o.inner, o.inner_cycles, o.outer = int(inner), int(inner_cycles), int(outer)
        o.inner_krylov, o.check_every = int(inner_krylov), int(check_every)
        self._gv, self._gp = vgrid.c(torch.float64), pgrid.c(torch.float64)
        self.fp = fp
        h = ctypes.c_void_p(0)
        _check(lib().nn4_flow_create(ctypes.byref(self._gv), ctypes.byref(self._gp), ctypes.byref(fp),
                                     ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def step(self, C, u, v, w, p_hs, p_nh, stream=None):
        st = _FlowStats()
        _check(lib().nn4_flow_step(self._h, _ptr(C), _ptr(u), _ptr(v), _ptr(w), _ptr(p_hs), _ptr(p_nh),
                                   ctypes.byref(st), _stream(stream)))
        return {"mass": st.mass, "c_min": st.c_min, "c_max": st.c_max, "hs_iters": st.hs_iters,
                "nh_iters": st.nh_iters, "hs_rel": st.hs_rel, "nh_rel": st.nh_rel}

    def close(self):
        if self._h is not None and self._h.value:
            lib().nn4_flow_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
