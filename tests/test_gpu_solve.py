"""GPU parity of the V-cycle and the pressure solves against the FP64 oracle.

* plain FP64: every V-cycle agrees with the oracle's cycle to 1e-12 relative (the oracle runs
  the same sawtooth cycle), and the solve's residual history agrees to 1e-12;
* mixed precision (FP32 / BF16 storage, FP64 outer loop): the solution agrees with the oracle's
  converged FP64 solution of A x = b to 1e-8 relative (after removing the mean for the singular
  all-natural problem);
* flexible CG with Galerkin coarse operators for a 1000:1 density sphere: FP64 per-iteration
  parity with the oracle's flexible CG, mixed-precision solution error <= 1e-8.
"""

import numpy as np
import pytest
import torch

from oracle import direct, fem, mg
from synth import sphere_ramp_field, standard_normal, uniform01
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _nn4():
    from paper_2401_06755_gb300 import nn4
    return nn4


def _grids(n, h, bc):
    nn4 = _nn4()
    g = mg.Grid(tuple(n), tuple(h), tuple(bc))
    G = nn4.Grid(tuple(n), tuple(h), tuple(nn4.DIRICHLET if d else nn4.NATURAL for d in bc))
    return g, G


def _rhs(g, seed):
    b = fem.lumped_mass(g.shape, g.h) * standard_normal(seed, int(np.prod(g.shape))).reshape(g.shape)
    b[mg.dirichlet_mask(g)] = 0.0
    if mg.is_singular(g):
        b -= b.mean()
    return b


def _sphere_k(g, seed=0, ratio=1000.0):
    c = 0.3 + 0.4 * uniform01(seed, 3)
    C = sphere_ramp_field(g.n, g.h, c, 0.2, 2 * max(g.h))
    return 1.0 / (ratio * C + (1.0 - C))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CYCLE_CASES = [
    ((33, 33, 33), (1 / 32,) * 3, (True,) * 6, False),
    ((17, 9, 33), (1 / 16, 1 / 8, 1 / 32), (False,) * 5 + (True,), False),
    ((33, 17, 17), (1 / 32, 1 / 16, 1 / 16), (False,) * 6, False),
    ((17, 17, 17), (1 / 16,) * 3, (False,) * 6, True),
    ((17, 9, 17), (1 / 16, 1 / 8, 1 / 16), (False,) * 5 + (True,), True),
    ((3, 3, 3), (0.5,) * 3, (True,) * 6, False),
    # Galerkin levels of 32 m + 1 columns (the tiled 27-point pass's extra last column), several x
    # tiles and z chunks: 65 x 33 x 17 and 33 x 17 x 9 below 129 x 65 x 33.  The larger case runs
    # at a 10:1 sphere: at 1000:1 the FP64 cycles of this grid and the oracle's drift apart by
    # 7.5e-13 per cycle (rounding of the two triple products, amplified by the coarse correction;
    # the same before and after the 27-point pass was tiled), which the 1e-12 bound cannot absorb.
    ((129, 65, 33), (1 / 128, 1 / 64, 1 / 32), (False, True, False, False, False, True), 10.0),
    ((65, 33, 17), (1 / 64, 1 / 32, 1 / 16), (True, False, False, False, True, False), True),
]


@pytest.mark.parametrize("ci", range(len(CYCLE_CASES)))
def test_vcycle_fp64_per_cycle(ci):
    """nn4_vcycle on FP64 arrays reproduces the oracle's sawtooth cycle to 1e-12 per cycle."""
    need_gpu()
    nn4 = _nn4()
    n, h, bc, vc = CYCLE_CASES[ci]
    g, G = _grids(n, h, bc)
    k = (_sphere_k(g) if vc is True else _sphere_k(g, ratio=vc)) if vc else None
    b = _rhs(g, 1 + ci)
    lv = mg.Levels(g, k)
    K = nn4.to_field(k, G) if vc else None
    plans = [nn4.Plan(G, K), nn4.Plan(G, K, coarse_tail=False)]
    B = nn4.to_field(b, G)
    Xs = [nn4.field(G), nn4.field(G)]
    x = np.zeros(g.shape)
    for c in range(6):
        x = mg.vcycle(lv, x, b)
        for plan, X in zip(plans, Xs):
            plan.vcycle(B, X)
            xg = nn4.nodes(X, G).cpu().numpy()
            assert _rel(xg, x) <= 1e-12, f"cycle {c}: {_rel(xg, x):.3e}"


@pytest.mark.parametrize("shape", range(5))
def test_every_tile_shape(shape):
    """Each compiled tile shape of the stencil pass, forced on every pass of a plan, gives the
    oracle's FP64 cycle to 1e-12 and a mixed FP32 flexible-CG solve (fused dot, precomputed 1/D)
    within 1e-8 of the oracle's converged solution.  Eq. k-T with a 1000:1 sphere, Dirichlet on two
    faces, sizes that leave ragged tiles along every axis; the coarse levels run in the cooperative
    launch with the dense tail map."""
    need_gpu()
    nn4 = _nn4()
    assert nn4.pass_shapes() == 5
    bc = (False, False, True, False, False, True)
    g, G = _grids((33, 17, 49), (1 / 32,) * 3, bc)
    k = _sphere_k(g)
    b = _rhs(g, 11)
    K = nn4.to_field(k, G)
    lv = mg.Levels(g, k)
    plan = nn4.Plan(G, K, pass_shape=shape)
    B, X = nn4.to_field(b, G), nn4.field(G)
    x = np.zeros(g.shape)
    for c in range(3):
        x = mg.vcycle(lv, x, b)
        plan.vcycle(B, X)
        assert _rel(nn4.nodes(X, G).cpu().numpy(), x) <= 1e-12, f"cycle {c}"
    xref, _ = mg.pressure_solve_fcg(g, b, k=k, rtol=1e-13, max_iters=200)
    mixed = nn4.Plan(G, K, inner=nn4.F32, outer=nn4.OUTER_FCG, inner_krylov=6, pass_shape=shape)
    X2 = nn4.field(G)
    info = mixed.solve(B, X2, rtol=1e-11, max_iters=60)
    assert info["status"] == nn4.OK
    assert _rel(nn4.nodes(X2, G).cpu().numpy(), xref) <= 1e-8


@pytest.mark.parametrize("inner", ["f64", "f32", "bf16"])
def test_fused_prolongation_matches_separate_launch(inner):
    """The level-0 sweep that forms the prolonged correction from coarse tiles gives the solve of
    the separate prolongation launch: FP64 histories and solutions agree to 1e-12 (rounding: the
    same operations, contracted differently), FP32/BF16 to 1e-5 (histories: plus 1e-9 absolute).
    Mixed faces, ragged sizes."""
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((65, 33, 49), (1 / 64,) * 3, (True, False, False, False, False, True))
    k = _sphere_k(g)
    b = _rhs(g, 13)
    K, B = nn4.to_field(k, G), nn4.to_field(b, G)
    dt = {"f64": nn4.F64, "f32": nn4.F32, "bf16": nn4.BF16}[inner]
    out = []
    for fused in (True, False):
        plan = nn4.Plan(G, K, inner=dt, outer=nn4.OUTER_FCG, inner_krylov=0 if inner == "f64" else 4,
                        fused_prolong=fused, autotune=False)
        X = nn4.field(G)
        info = plan.solve(B, X, rtol=0.0, max_iters=5)
        out.append((np.array(info["history"]), nn4.nodes(X, G).cpu().numpy()))
    # FP32/BF16: the inner reductions use atomics, so runs differ at the FP32 noise floor of the
    # relative residual (~1e-11 absolute at 1e-7): a relative bound plus an absolute floor
    tol, floor = (1e-12, 0.0) if inner == "f64" else (1e-5, 1e-9)
    assert np.all(np.abs(out[0][0] - out[1][0]) <= tol * out[1][0] + floor)
    assert _rel(out[0][1], out[1][1]) <= tol


def test_solve_fp64_fixed_cycles_history():
    """Config-1 style: 33^3 Dirichlet, 20 cycles; history and solution match the oracle."""
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((33,) * 3, (1 / 32,) * 3, (True,) * 6)
    b = fem.lumped_mass(g.shape, g.h) * standard_normal(0, 33 ** 3).reshape(g.shape)
    b[mg.dirichlet_mask(g)] = 0.0
    xo, ho = mg.pressure_solve(g, b, fixed_cycles=20)
    for graph in (True, False):
        plan = nn4.Plan(G, use_graph=graph)
        B, X = nn4.to_field(b, G), nn4.field(G)
        info = plan.solve(B, X, rtol=0.0, max_iters=20)
        assert info["iterations"] == 20
        hg = np.array(info["history"])
        assert np.all(np.abs(hg - np.array(ho)) <= 1e-12 * np.maximum(hg, 1e-3))
        assert _rel(nn4.nodes(X, G).cpu().numpy(), xo) <= 1e-12


@pytest.mark.parametrize("outer", ["cycles", "fcg"])
def test_solve_fp64_warm_start(outer):
    """A nonzero initial guess (also on Dirichlet nodes, which enter A x0 at their neighbours)
    takes the residual path; a zero one the copy path: both match the oracle."""
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((33, 17, 33), (1 / 32,) * 3, (True, False, False, False, True, True))
    b = _rhs(g, 5)
    b[mg.dirichlet_mask(g)] = 0.0
    x0 = 0.1 * standard_normal(6, int(np.prod(g.shape))).reshape(g.shape)
    for start in (x0, np.zeros(g.shape)):
        if outer == "cycles":
            xo, ho = mg.pressure_solve(g, b, x0=start, fixed_cycles=8)
            plan = nn4.Plan(G)
            iters = 8
        else:
            xo, ho = mg.pressure_solve_fcg(g, b, x0=start, rtol=0.0, max_iters=6)
            plan = nn4.Plan(G, outer=nn4.OUTER_FCG)
            iters = 6
        B, X = nn4.to_field(b, G), nn4.to_field(start, G)
        info = plan.solve(B, X, rtol=0.0, max_iters=iters)
        hg = np.array(info["history"])
        assert np.all(np.abs(hg - np.array(ho[:len(hg)])) <= 1e-12 + 1e-9 * np.array(ho[:len(hg)]))
        assert _rel(nn4.nodes(X, G).cpu().numpy(), xo) <= 1e-11


@pytest.mark.parametrize("inner", ["f32", "bf16"])
@pytest.mark.parametrize("outer", ["cycles", "fcg"])
def test_solve_mixed_constant_coefficient(inner, outer):
    need_gpu()
    nn4 = _nn4()
    # isotropic spacing: point Jacobi with full coarsening is only efficient without anisotropy
    g, G = _grids((65, 33, 33), (1 / 64,) * 3, (False,) * 5 + (True,))
    b = _rhs(g, 4)
    xref = direct.solve_cg(g, b, rtol=1e-14)
    plan = nn4.Plan(G, inner=nn4.F32 if inner == "f32" else nn4.BF16, inner_cycles=2,
                    outer=nn4.OUTER_CYCLES if outer == "cycles" else nn4.OUTER_FCG)
    B, X = nn4.to_field(b, G), nn4.field(G)
    info = plan.solve(B, X, rtol=1e-11, max_iters=200)
    assert info["status"] == nn4.OK and info["rel_res"] <= 1e-11
    assert _rel(nn4.nodes(X, G).cpu().numpy(), xref) <= 1e-8


def test_fcg_fp64_matches_oracle_sphere():
    """Flexible CG + Galerkin cycle at 33^3, 1000:1 sphere, all-natural: FP64 per-iteration
    residual history matches the oracle's; the solution matches the dense-free CG reference."""
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((33,) * 3, (1 / 32,) * 3, (False,) * 6)
    k = _sphere_k(g)
    b = _rhs(g, 1)
    xo, ho = mg.pressure_solve_fcg(g, b, k=k, rtol=1e-10, max_iters=80)
    plan = nn4.Plan(G, nn4.to_field(k, G), outer=nn4.OUTER_FCG)
    B, X = nn4.to_field(b, G), nn4.field(G)
    info = plan.solve(B, X, rtol=1e-10, max_iters=80)
    hg = np.array(info["history"])
    m = min(len(hg), len(ho))
    # relative residuals (units of ||b||) agree to 1e-12: the FP64 rounding of the recurrence
    assert np.all(np.abs(hg[:m] - np.array(ho[:m])) <= 1e-12 + 1e-9 * np.array(ho[:m]))
    xg = nn4.nodes(X, G).cpu().numpy()
    assert _rel(xg - xg.mean(), xo - xo.mean()) <= 1e-9


@pytest.mark.parametrize("inner", ["f32", "bf16"])
def test_fcg_mixed_sphere_error(inner):
    """Precision form at 65^3: mixed flexible CG reaches the FP64 solution to <= 1e-8."""
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((65,) * 3, (1 / 64,) * 3, (False,) * 6)
    k = _sphere_k(g)
    b = _rhs(g, 1)
    xref, _ = mg.pressure_solve_fcg(g, b, k=k, rtol=1e-13, max_iters=200)
    plan = nn4.Plan(G, nn4.to_field(k, G), inner=nn4.F32 if inner == "f32" else nn4.BF16,
                    inner_cycles=2, outer=nn4.OUTER_FCG)
    B, X = nn4.to_field(b, G), nn4.field(G)
    info = plan.solve(B, X, rtol=1e-10, max_iters=200)
    assert info["status"] == nn4.OK
    xg = nn4.nodes(X, G).cpu().numpy()
    m = fem.lumped_mass(g.shape, g.h)
    mean = lambda v: (m * v).sum() / m.sum()
    assert _rel(xg - mean(xg), xref - mean(xref)) <= 1e-8


def test_host_buffers_equal_device_solve():
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((33, 17, 17), (1 / 32, 1 / 16, 1 / 16), (False,) * 5 + (True,))
    b = _rhs(g, 9)
    plan = nn4.Plan(G, inner=nn4.F32, inner_cycles=2)
    B, X = nn4.to_field(b, G), nn4.field(G)
    i1 = plan.solve(B, X, rtol=1e-10)
    bh = torch.tensor(b).contiguous().pin_memory()
    xh = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
    i2 = plan.solve_host(bh, xh, rtol=1e-10)
    assert i1["iterations"] == i2["iterations"]
    np.testing.assert_array_equal(nn4.nodes(X, G).cpu().numpy(), xh.numpy())


def test_error_paths():
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((17,) * 3, (1 / 16,) * 3, (True,) * 6)
    plan = nn4.Plan(G)
    b = _rhs(g, 2)
    b[5, 5, 5] = np.nan
    with pytest.raises(nn4.NN4Error) as e:
        plan.solve(nn4.to_field(b, G), nn4.field(G), rtol=1e-8)
    assert e.value.code == nn4.ENONFINITE
    b = _rhs(g, 2)
    info = plan.solve(nn4.to_field(b, G), nn4.field(G), rtol=1e-14, max_iters=3)
    assert info["status"] == nn4.ENOCONV and info["iterations"] == 3
    assert nn4.device_error() == nn4.OK


@pytest.mark.parametrize("inner", ["f32", "bf16"])
def test_inner_krylov_sphere_error(inner):
    """Precision form with the FP32 inner flexible-CG loop: few FP64 outer iterations, the
    solution agrees with the FP64 oracle's to <= 1e-8 (means removed)."""
    need_gpu()
    nn4 = _nn4()
    g, G = _grids((65,) * 3, (1 / 64,) * 3, (False,) * 6)
    k = _sphere_k(g)
    b = _rhs(g, 1)
    xref, _ = mg.pressure_solve_fcg(g, b, k=k, rtol=1e-13, max_iters=200)
    plan = nn4.Plan(G, nn4.to_field(k, G), inner=nn4.F32 if inner == "f32" else nn4.BF16,
                    inner_cycles=1, outer=nn4.OUTER_FCG, inner_krylov=12)
    B, X = nn4.to_field(b, G), nn4.field(G)
    info = plan.solve(B, X, rtol=1e-10, max_iters=50)
    assert info["status"] == nn4.OK and info["iterations"] <= 10
    xg = nn4.nodes(X, G).cpu().numpy()
    m = fem.lumped_mass(g.shape, g.h)
    mean = lambda v: (m * v).sum() / m.sum()
    assert _rel(xg - mean(xg), xref - mean(xref)) <= 1e-8
    # defect-correction outer loop with the same inner loop
    plan2 = nn4.Plan(G, nn4.to_field(k, G), inner=nn4.F32, inner_cycles=1, outer=nn4.OUTER_CYCLES,
                     inner_krylov=12)
    X2 = nn4.field(G)
    info2 = plan2.solve(B, X2, rtol=1e-10, max_iters=50)
    assert info2["status"] == nn4.OK
    xg2 = nn4.nodes(X2, G).cpu().numpy()
    assert _rel(xg2 - mean(xg2), xref - mean(xref)) <= 1e-8


def test_full_size_mixed_solve_in_the_timed_configuration():
    """The timed configuration at its full size: the 257^3 precision-form workload (k = 1/rho at a
    1000:1 density ratio, all faces natural) with the benchmark's plan (FP32 hierarchy, 10 FP32
    flexible-CG iterations per FP64 flexible-CG iteration).  The oracle recomputes the relative
    residual of the returned solution on the host, a property that holds at any size; it must
    meet the tolerance and agree with the residual the solve reports."""
    need_gpu()
    import bench
    nn4 = _nn4()
    n = 257
    h, k, b = bench.workload(n)
    G = nn4.Grid((n,) * 3, (h,) * 3)
    plan = nn4.Plan(G, nn4.to_field(k, G), inner=nn4.F32, inner_cycles=1, outer=nn4.OUTER_FCG,
                    check_every=1, inner_krylov=10)
    X = nn4.field(G)
    info = plan.solve(nn4.to_field(b, G), X, rtol=1e-8, max_iters=400)
    assert info["status"] == nn4.OK
    x = nn4.nodes(X, G).cpu().numpy()
    del X
    plan.close()
    g = mg.Grid((n,) * 3, (h,) * 3)
    rel = float(np.linalg.norm(mg.residual(g, b, x, k)) / np.linalg.norm(b))
    assert rel <= 1e-8, rel
    assert abs(rel - info["rel_res"]) <= 1e-12 + 1e-3 * rel, (rel, info["rel_res"])


def test_mixed_solve_at_129_matches_oracle_solution():
    """The timed configuration (FP32 hierarchy, 10 FP32 flexible-CG iterations per FP64
    flexible-CG iteration, rtol 1e-8) on the precision-form workload at 129^3, the largest size
    the oracle solves in minutes: the GPU solution agrees with the oracle's flexible-CG solution
    converged to 1e-12 to <= 1e-8 relative, means (lumped-mass weighted) removed.  The oracle
    runs on the host for about three minutes."""
    need_gpu()
    import bench
    nn4 = _nn4()
    n = 129
    h, k, b = bench.workload(n)
    G = nn4.Grid((n,) * 3, (h,) * 3)
    plan = nn4.Plan(G, nn4.to_field(k, G), inner=nn4.F32, inner_cycles=1, outer=nn4.OUTER_FCG,
                    check_every=1, inner_krylov=10)
    X = nn4.field(G)
    info = plan.solve(nn4.to_field(b, G), X, rtol=1e-8, max_iters=400)
    assert info["status"] == nn4.OK
    xg = nn4.nodes(X, G).cpu().numpy()
    plan.close()
    g = mg.Grid((n,) * 3, (h,) * 3)
    xref, hist = mg.pressure_solve_fcg(g, b, k=k, rtol=1e-12, max_iters=80)
    assert hist[-1] <= 1e-12, hist[-1]
    m = fem.lumped_mass(g.shape, g.h)
    mean = lambda v: (m * v).sum() / m.sum()
    err = _rel(xg - mean(xg), xref - mean(xref))
    print(f"PARITY solve129.mixed_vs_oracle {err:.3e} (tol 1.0e-08)")
    assert err <= 1e-8, err
