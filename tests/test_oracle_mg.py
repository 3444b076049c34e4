"""Pins of the oracle's multigrid against direct solves, convergence order and invariants."""

import numpy as np
import pytest

from oracle import direct, fem, mg
from synth import node_coords, standard_normal


def _rhs(g, seed):
    b = fem.lumped_mass(g.shape, g.h) * standard_normal(seed, int(np.prod(g.shape))).reshape(g.shape)
    b[mg.dirichlet_mask(g)] = 0.0
    if mg.is_singular(g):
        b -= b.mean()
    return b


def test_coarsening_schedule():
    sizes = lambda n: [G.n for G in mg.hierarchy(mg.Grid(n, (1.0, 1.0, 1.0)))]
    assert sizes((33,) * 3) == [(33,) * 3, (17,) * 3, (9,) * 3, (5,) * 3, (3,) * 3]
    assert len(sizes((257,) * 3)) == 8
    assert sizes((97,) * 3)[-1] == (4, 4, 4)
    assert sizes((129, 65, 65))[-1] == (5, 3, 3)


def test_prolongation_exact_for_trilinear_fields():
    """P reproduces any trilinear function exactly (it is Q1 interpolation)."""
    gf = mg.Grid((9, 5, 17), (0.1, 0.2, 0.05))
    gc = gf.coarse()
    xf, yf, zf = node_coords(gf.n, gf.h)
    xc, yc, zc = node_coords(gc.n, gc.h)
    f = lambda x, y, z: 1 + 2 * x - y + 3 * z + x * y - 2 * y * z + x * y * z
    np.testing.assert_allclose(mg.prolong_raw(gc, f(xc, yc, zc)), f(xf, yf, zf), atol=1e-14)


@pytest.mark.parametrize("n,bc", [
    (5, (True,) * 6),
    (9, (True,) * 6),
    (9, (False,) * 5 + (True,)),
    (9, (False,) * 6),
    (5, (False,) * 6),
])
def test_vcycle_converges_to_dense_solution(n, bc):
    """V-cycles iterated to 1e-14 agree with dense LU to 1e-12 (zero mean when singular)."""
    g = mg.Grid((n, n, n), (1.0 / (n - 1),) * 3, bc)
    b = _rhs(g, 7)
    x, hist = mg.pressure_solve(g, b, rtol=1e-14, max_cycles=300)
    assert hist[-1] <= 1e-14
    xd = direct.solve_dense(g, b)
    if mg.is_singular(g):
        x = x - x.mean()
        xd = xd - xd.mean()
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_vcycle_variable_coefficient_matches_dense():
    g = mg.Grid((9, 9, 9), (0.125,) * 3, (False,) * 5 + (True,))
    k = 1.0 / (1.0 + 9.0 * (standard_normal(5, 729).reshape(g.shape) > 0.5))
    b = _rhs(g, 11)
    x, hist = mg.pressure_solve(g, b, k=k, rtol=1e-14, max_cycles=500)
    xd = direct.solve_dense(g, b, k)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_cg_matches_dense():
    g = mg.Grid((9, 5, 9), (0.125, 0.25, 0.125), (True,) * 6)
    b = _rhs(g, 2)
    np.testing.assert_allclose(direct.solve_cg(g, b), direct.solve_dense(g, b), atol=1e-13)


def test_manufactured_solution_second_order():
    """p = sin(pi x) sin(pi y) sin(pi z), f = 3 pi^2 p: nodal max error is O(h^2)."""
    errs = []
    ns = [9, 17, 33]
    for n in ns:
        h = 1.0 / (n - 1)
        g = mg.Grid((n, n, n), (h, h, h), (True,) * 6)
        x, y, z = node_coords(g.n, g.h)
        p = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        b = fem.lumped_mass(g.shape, g.h) * 3 * np.pi**2 * p
        b[mg.dirichlet_mask(g)] = 0.0
        sol, _ = mg.pressure_solve(g, b, rtol=1e-13, max_cycles=200)
        errs.append(np.abs(sol - p).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(1.9 <= o <= 2.1 for o in orders), orders


def test_constant_field_zero_residual_and_hydrostatic_line():
    """A.1 = 0 on natural rows; a linear field is reproduced exactly by the solve."""
    g = mg.Grid((9, 9, 9), (0.125,) * 3, (False,) * 5 + (True,))
    r = mg.residual(g, np.zeros(g.shape), np.ones(g.shape))
    assert np.abs(r).max() < 1e-14
    # linear p = 1 - z with zero source: the natural boundary flux of the linear field is the
    # only right-hand side; b = A p; the solve from zero with p fixed at the Dirichlet top
    _, _, z = node_coords(g.n, g.h)
    p = 1.0 - z
    b = mg.stencil_apply(g, p)
    b[mg.dirichlet_mask(g)] = 0.0
    sol, _ = mg.pressure_solve(g, b, rtol=1e-14, max_cycles=300)
    assert np.abs(sol - p).max() < 1e-12


def test_jacobi_symbol_values():
    """Weighted Jacobi on Fourier modes, from the symbols of K1 = [-1,2,-1]/h, M1 = h[1,4,1]/6.

    D^-1 A has symbol 3/2 on the face mode (pi,0,0), 1 on (pi,pi,0) and 1/2 on the checkerboard
    (pi,pi,pi); with omega = 2/3 one sweep multiplies them by 0, 1/3 and 2/3 at nodes that do not
    see the boundary.  (2/3 is the smoothing factor of the cycle.)
    """
    n = 17
    g = mg.Grid((n, n, n), (1 / 16,) * 3, (True,) * 6)
    iz, iy, ix = np.indices(g.shape)
    for mode, factor in (((ix,), 0.0), ((ix, iy), 1 / 3), ((ix, iy, iz), 2 / 3)):
        e = (-1.0) ** sum(mode)
        e = np.where(mg.dirichlet_mask(g), 0.0, e)
        e1 = mg.jacobi(g, np.zeros(g.shape), e)
        inner = (slice(2, -2),) * 3
        np.testing.assert_allclose(e1[inner], factor * e[inner], atol=1e-13)


def test_pressure_solve_history_monotone():
    n = 17
    g = mg.Grid((n, n, n), (1 / 16,) * 3, (True,) * 6)
    b = _rhs(g, 0)
    _, hist = mg.pressure_solve(g, b, fixed_cycles=10)
    assert len(hist) == 11 and all(hist[i + 1] < hist[i] for i in range(10))


def _sphere_k(g, ratio=1000.0, seed=0):
    from synth import sphere_ramp_field, uniform01
    c = 0.3 + 0.4 * uniform01(seed, 3)
    C = sphere_ramp_field(g.n, g.h, c, 0.2, 2 * max(g.h))
    return 1.0 / (ratio * C + (1.0 - C))


def test_sparse_operator_matches_matrix_free():
    rng = np.random.default_rng(1)
    g = mg.Grid((9, 5, 7), (0.1, 0.3, 0.2), (True, False, False, True, False, False))
    k = np.exp(rng.standard_normal(g.shape))
    x = rng.standard_normal(g.shape)
    A = mg.sparse_operator(g, k)
    np.testing.assert_allclose((A @ x.ravel()).reshape(g.shape), mg.stencil_apply(g, x, k),
                               atol=1e-13)


def test_galerkin_coarse_operator_is_dense_triple_product():
    """The sparse Galerkin product equals P^T A P built column by column from the matrix-free
    operator and the masked prolongation (variable coefficient, mixed boundary faces)."""
    rng = np.random.default_rng(4)
    g = mg.Grid((9, 9, 5), (0.125, 0.125, 0.25), (False,) * 5 + (True,))
    k = np.exp(2 * rng.standard_normal(g.shape))
    lv = mg.Levels(g, k)
    gc = g.coarse()
    Af, ff = mg.dense_matrix(g, k)
    fc = np.flatnonzero(~mg.dirichlet_mask(gc).ravel())
    P = np.zeros((ff.size, fc.size))
    for c, j in enumerate(fc):
        e = np.zeros(gc.shape)
        e.ravel()[j] = 1.0
        P[:, c] = mg.prolong(g, e).ravel()[ff]
    Ac = lv.A[1].toarray()[np.ix_(fc, fc)]
    np.testing.assert_allclose(Ac, P.T @ Af @ P, atol=1e-13 * np.abs(Ac).max())
    # symmetric with zero row sums on natural rows away from the Dirichlet face
    np.testing.assert_allclose(Ac, Ac.T, atol=1e-14 * np.abs(Ac).max())


@pytest.mark.parametrize("bc", [(False,) * 6, (False,) * 5 + (True,)])
def test_fcg_matches_dense_sphere(bc):
    """Flexible CG with V-cycle preconditioning reaches the dense solution (1000:1 sphere)."""
    n = 9
    g = mg.Grid((n, n, n), (1.0 / (n - 1),) * 3, bc)
    k = _sphere_k(g)
    b = _rhs(g, 3)
    for m in (1, 2):
        x, hist = mg.pressure_solve_fcg(g, b, k=k, rtol=1e-13, max_iters=200, inner_cycles=m)
        assert hist[-1] <= 1e-13
        xd = direct.solve_dense(g, b, k)
        if mg.is_singular(g):
            x = x - x.mean()
            xd = xd - xd.mean()
        assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)


def test_fcg_sphere_33_converges_fast():
    """At 33^3 with a 1000:1 sphere the Galerkin cycle inside flexible CG reaches 1e-8 in
    well under 40 iterations (the plain repeated cycle needs far more)."""
    n = 33
    g = mg.Grid((n, n, n), (1.0 / (n - 1),) * 3)
    k = _sphere_k(g)
    b = _rhs(g, 1)
    _, hist = mg.pressure_solve_fcg(g, b, k=k, rtol=1e-8, max_iters=60)
    assert hist[-1] <= 1e-8 and len(hist) - 1 <= 40
    _, hist_plain = mg.pressure_solve(g, b, k=k, fixed_cycles=12)
    assert hist_plain[-1] > 1e-6


def test_min_norm_coarsest_solve_high_contrast():
    """The singular coarsest solve returns the zero-mean solution even when the null
    eigenvalue is at rounding level (1000:1 sphere, Galerkin 3^3 level)."""
    n = 17
    g = mg.Grid((n,) * 3, (1 / 16,) * 3)
    lv = mg.Levels(g, _sphere_k(g))
    A = lv.A[-1].toarray()
    r = np.random.default_rng(0).standard_normal(A.shape[0])
    r -= r.mean()
    e = mg.min_norm_solve(A, r)
    assert abs(e.mean()) < 1e-10 * np.abs(e).max()
    np.testing.assert_allclose(A @ e, r, atol=1e-9 * np.abs(r).max())
