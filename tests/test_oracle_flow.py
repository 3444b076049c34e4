"""Pins of the oracle's explicit flow terms: printed constants, exact quadrature, invariants."""

import os

import numpy as np

from oracle import fem, flow
from synth import node_coords, sphere_ramp_field

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_constants_match_printed_values():
    prm = flow.VOFParams()
    for line in open(os.path.join(GOLDEN, "vof_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, value = line.split()[:2]
        if name == "alpha_ksquare":
            assert 8.0 / 2 ** prm.p == float(value)
            continue
        assert getattr(prm, name) == float(value), name


def test_mass_sum_is_exact_quadrature():
    """Lumped nodal volumes integrate constants and trilinear fields exactly (trapezoid rule)."""
    n, h = (9, 5, 7), (0.25, 0.5, 1 / 6)
    L = [(m - 1) * hh for m, hh in zip(n, h)]
    x, y, z = node_coords(n, h)
    assert abs(flow.mass_sum(x.shape, h, np.ones(x.shape)) - L[0] * L[1] * L[2]) < 1e-14
    f = 1 + 2 * x + 3 * y * z
    exact = L[0] * L[1] * L[2] + L[0] ** 2 * L[1] * L[2] + 3 * L[0] * (L[1] ** 2 / 2) * (L[2] ** 2 / 2)
    assert abs(flow.mass_sum(x.shape, h, f) - exact) < 1e-13


def test_uniform_field_stays_uniform():
    n, h = (9, 7, 8), (0.1, 0.1, 0.1)
    rng = np.random.default_rng(0)
    shape = (n[2], n[1], n[0])
    for c0 in (0.5, 0.97, 0.01):
        C = np.full(shape, c0)
        u, v, w = (rng.standard_normal(shape) for _ in range(3))
        s, Cn, parts = flow.vof_step(shape, h, C, u, v, w, 1e-3)
        assert np.abs(s).max() < 1e-14 and np.abs(Cn - c0).max() < 1e-14
        for k in parts["k"]:
            assert np.abs(k).max() < 1e-20  # rounding level of a zero gradient


def test_linear_profile_has_no_positive_weight():
    """C linear in x inside [0.05, 0.95]: S^x > 0 inside, so w^{x+} = 0 and w^{x-} = 1 there."""
    n, h = (11, 5, 5), (0.1, 0.1, 0.1)
    x, _, _ = node_coords(n, h)
    C = 0.1 + 0.8 * x
    shape = C.shape
    zeros = np.zeros(shape)
    _, _, parts = flow.vof_step(shape, h, C, zeros + 1.0, zeros, zeros, 1e-3)
    inner = (slice(None), slice(None), slice(1, -1))
    assert np.all(parts["w_plus"][0][inner] == 0.0)
    assert np.all(parts["w_minus"][0][inner] == 1.0)
    # the copy-halo makes S vanish on the x walls: no weight at all there
    assert np.all(parts["S"][0][:, :, 0] == 0.0) and np.all(parts["w_minus"][0][:, :, 0] == 0.0)


def test_invariant_direction_advection_leaves_interior_unchanged():
    """C varies along x only, u = (0, 1, 0): no advection, and constant-in-x diffusion
    coefficients acting on a linear profile vanish away from the walls."""
    n, h = (13, 9, 6), (0.05, 0.05, 0.05)
    x, _, _ = node_coords(n, h)
    C = 0.2 + 0.6 * x / x.max()
    shape = C.shape
    zeros = np.zeros(shape)
    s, Cn, parts = flow.vof_step(shape, h, C, zeros, zeros + 1.0, zeros, 1e-4)
    assert np.abs(parts["a_C"]).max() < 1e-12
    inner = (slice(None), slice(None), slice(2, -2))
    np.testing.assert_allclose(Cn[inner], C[inner], atol=1e-12)


def test_pure_advection_of_smooth_field_is_consistent():
    """A smooth field advected by a uniform velocity: the step matches C - dt u.grad C to O(h^2)
    in the interior (the Petrov-Galerkin terms are of higher order there)."""
    errs = []
    for nn in (17, 33):
        h = 1.0 / (nn - 1)
        n = (nn, nn, nn)
        x, y, z = node_coords(n, (h, h, h))
        C = 0.5 + 0.3 * np.sin(np.pi * x) * np.cos(np.pi * y)
        shape = C.shape
        u = np.full(shape, 0.3)
        v = np.full(shape, -0.2)
        w = np.zeros(shape)
        dt = 1e-3
        _, Cn, _ = flow.vof_step(shape, (h, h, h), C, u, v, w, dt)
        exact_rate = 0.3 * 0.3 * np.pi * np.cos(np.pi * x) * np.cos(np.pi * y) \
            - 0.2 * (-0.3 * np.pi) * np.sin(np.pi * x) * np.sin(np.pi * y)
        inner = (slice(3, -3),) * 3
        errs.append(np.abs((C - Cn)[inner] / dt - exact_rate[inner]).max())
    assert errs[1] < errs[0] / 2.5


def test_hydrostatic_column_is_exact():
    """Uniform density, no surface tension: the Stage-1 solve gives p = rho g (L - z) exactly
    (a linear field lies in the Q1 space; the natural bottom row imposes dp/dz = -rho g)."""
    from oracle import direct, mg
    n, h = (5, 5, 9), (0.25, 0.25, 0.125)
    g = mg.Grid(n, h, (False,) * 5 + (True,))
    prm = flow.FlowParams(sigma_t=0.0)
    C = np.full(g.shape, 1.0)
    b = flow.pressure_rhs_hydrostatic(g.shape, h, C, prm, mg.dirichlet_mask(g))
    p = direct.solve_dense(g, b)
    _, _, z = node_coords(n, h)
    np.testing.assert_allclose(p, prm.rho_l * prm.g * (z.max() - z), atol=1e-10)


def test_surface_tension_of_a_plane_interface_vanishes():
    """A planar interface (C linear in x) has zero curvature at interior nodes."""
    n, h = (9, 6, 6), (0.1, 0.1, 0.1)
    x, _, _ = node_coords(n, h)
    C = np.clip(0.2 + x, 0, 1)
    st, kappa = flow.surface_tension(C.shape, h, C, flow.FlowParams())
    assert np.abs(kappa[1:-1, 1:-1, 1:-1]).max() < 1e-8


def test_correction_rhs_vanishes_for_divergence_free_uniform_density():
    """Uniform rho and a divergence-free u~ = (y, -x, 0): the Stage-3 RHS is zero inside
    (the two filter terms cancel exactly for uniform rho; div u~ = 0)."""
    n, h = (7, 7, 7), (0.1, 0.1, 0.1)
    x, y, _ = node_coords(n, h)
    rho = np.full(x.shape, 3.0)
    b = flow.pressure_rhs_correction(x.shape, h, rho, [y, -x, np.zeros_like(x)], 1e-3)
    assert np.abs(b[1:-1, 1:-1, 1:-1]).max() < 1e-10


def test_velocity_correction_of_linear_pressure():
    """dp = a x: du = -dt a / rho at interior nodes, dv = dw = 0."""
    n, h = (7, 6, 5), (0.2, 0.1, 0.3)
    x, _, _ = node_coords(n, h)
    rho = np.full(x.shape, 2.0)
    du = flow.velocity_correction(x.shape, h, rho, 4.0 * x, 0.01)
    np.testing.assert_allclose(du[0][1:-1, 1:-1, 1:-1], -0.01 * 4.0 / 2.0, rtol=1e-12)
    assert np.abs(du[1]).max() < 1e-13 and np.abs(du[2]).max() < 1e-13


def test_momentum_at_rest_in_hydrostatic_balance():
    """Fluid at rest with p = rho g (L - z) and uniform rho: buoyancy and pressure gradient
    cancel at interior nodes, so u~ = 0 there (s_w = -g rho against f(p; w_z))."""
    n, h = (6, 6, 9), (0.2, 0.2, 0.125)
    _, _, z = node_coords(n, h)
    prm = flow.FlowParams(sigma_t=0.0, mu_l=1e-3)
    C = np.ones(z.shape)
    p = prm.rho_l * prm.g * (z.max() - z)
    zero = [np.zeros(z.shape)] * 3
    ut, uh = flow.momentum_predict(z.shape, h, C, zero, zero, p, 1e-3, prm)
    for c in range(3):
        assert np.abs(ut[c][1:-1, 1:-1, 1:-1]).max() < 1e-9


def test_mass_conserved_in_divergence_free_wall_tangent_flow():
    """Twenty Stage-4 steps in the flow of the stream function psi = A sin^2(pi x) sin^2(pi z)
    (u = dpsi/dz, w = -dpsi/dx: divergence-free, zero with its gradient on every wall): the lumped
    mass of C is conserved to rounding.  The consistent-mass Galerkin advection term integrates to
    the boundary flux, which vanishes (a mistaken component, index or velocity in it breaks this),
    and the Petrov-Galerkin diffusion terms conserve with natural faces for any coefficient.
    (Boundedness is not pinned: with the linear oscillation detectors the scheme over/undershoots
    under sustained advection, as the paper notes for them.)"""
    from synth import sphere_ramp_field
    n, h = (33, 9, 33), (1 / 32,) * 3
    x, y, z = node_coords(n, h)
    A = 0.25
    u = A * np.sin(np.pi * x) ** 2 * 2 * np.pi * np.sin(np.pi * z) * np.cos(np.pi * z)
    w = -A * 2 * np.pi * np.sin(np.pi * x) * np.cos(np.pi * x) * np.sin(np.pi * z) ** 2
    v = np.zeros_like(u)
    C = sphere_ramp_field(n, h, (0.5, 0.125, 0.35), 0.2, 2 * h[0])
    dt = 0.2 * h[0] / max(np.abs(u).max(), np.abs(w).max())
    m0 = flow.mass_sum(C.shape, h, C)
    for _ in range(20):
        _, C, _ = flow.vof_step(C.shape, h, C, u, v, w, dt)
    assert abs(flow.mass_sum(C.shape, h, C) - m0) <= 1e-9 * m0



def test_momentum_predictor_advects_a_linear_field_exactly():
    """One Stage-2 iteration on a linear velocity u = a + B x in a uniform fluid (no gravity,
    pressure or interface): at nodes two or more away from every face the Petrov-Galerkin
    coefficient a_Psi vanishes (the consistent mass reproduces a linear g = u.grad Psi), the
    diffusion of a linear component vanishes, and the lumped first-derivative filters are exact,
    so u~_c = u_c - dt sum_d u_d B_cd exactly.  B is not symmetric, so a transposed gradient, a
    wrong component, a wrong sign or a missing rho / m normalisation fails."""
    n, h = (17, 13, 11), (1 / 16, 1 / 12, 1 / 10)
    x, y, z = node_coords(n, h)
    a = np.array([0.3, -0.2, 0.1])
    B = np.array([[0.5, 0.2, -0.1], [0.3, -0.4, 0.25], [-0.15, 0.35, 0.6]])
    X = (x, y, z)
    u = [a[c] + sum(B[c, d] * X[d] for d in range(3)) for c in range(3)]
    prm = flow.FlowParams(g=0.0)
    C = np.ones(x.shape)
    dt = 1e-3
    ut, uh = flow.momentum_predict(x.shape, h, C, u, u, np.zeros(x.shape), dt, prm)
    inner = (slice(2, -2),) * 3
    for c in range(3):
        expect = u[c] - dt * sum(u[d] * B[c, d] for d in range(3))
        assert np.abs(ut[c][inner] - expect[inner]).max() <= 1e-13, c
        assert np.allclose(uh[c], 0.5 * (u[c] + ut[c]), rtol=0, atol=1e-15)
    # the same field moves at the boundary too (the scheme is not exact there): a non-trivial check
    assert max(np.abs(ut[c] - u[c]).max() for c in range(3)) > 1e-5


def test_surface_tension_curvature_of_a_sphere():
    """Curvature of a smeared sphere (ramp of 8 nodes): n = grad C / |grad C| is the outward radial
    unit vector, so kappa = div n = 2 / r where the ramp covers every neighbour of a node.  A
    dropped axis would give about (2/3)(2/r) and a sign error -2/r."""
    n, h = (33, 33, 33), (1 / 32,) * 3
    centre, R, width = (0.5, 0.5, 0.5), 0.3, 8 / 32
    C = sphere_ramp_field(n, h, centre, R, width)
    prm = flow.FlowParams()
    st, kappa = flow.surface_tension(C.shape, h, C, prm)
    x, y, z = node_coords(n, h)
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    band = np.abs(r - R) <= 2 * h[0]  # at least two nodes inside the ramp on either side
    rel = np.abs(kappa[band] * r[band] / 2 - 1)
    assert band.sum() > 500
    assert np.median(rel) < 1e-3 and rel.max() < 0.02
    # s_t = sigma kappa grad C points along +r (C grows outward, kappa > 0)
    sr = (st[0] * (x - centre[0]) + st[1] * (y - centre[1]) + st[2] * (z - centre[2]))[band]
    assert np.all(sr > 0)


def _smooth_state(n, h):
    x, y, z = node_coords(n, h)
    C = sphere_ramp_field(n, h, (0.45, 0.55, 0.5), 0.3, 3 * h[0])
    u = 0.3 * np.sin(2 * x + 1) * np.cos(3 * y) * (1 + z)
    v = 0.2 * np.cos(x) * np.sin(2 * y + 0.5) * (1 - z)
    w = 0.1 * np.sin(x + y) * np.cos(z)
    return C, [u, v, w], z


_FLIP = {0: lambda a: a[:, :, ::-1], 1: lambda a: a[:, ::-1, :], 2: lambda a: a[::-1, :, :]}


def test_vof_step_is_mirror_and_axis_swap_symmetric():
    """The compressive scheme has no preferred direction: mirroring an axis (with its velocity
    component negated) mirrors s_C, and exchanging x and y (equal spacings, u and v exchanged)
    exchanges it, to rounding.  An index slip on one side of a stencil or detector (an upwind
    choice taken the wrong way, a one-sided difference) breaks this."""
    n, h = (17, 17, 13), (1 / 16, 1 / 16, 1 / 12)
    C, U, _ = _smooth_state(n, h)
    s, _, _ = flow.vof_step(C.shape, h, C, *U, 1e-3)
    scale = np.abs(s).max()
    for d, f in _FLIP.items():
        Um = [(-f(U[c]) if c == d else f(U[c])) for c in range(3)]
        sm, _, _ = flow.vof_step(C.shape, h, f(C), *Um, 1e-3)
        assert np.abs(f(sm) - s).max() <= 1e-12 * scale, d
    tr = lambda a: np.swapaxes(a, 1, 2)
    st, _, _ = flow.vof_step(C.shape, h, tr(C), tr(U[1]), tr(U[0]), tr(U[2]), 1e-3)
    assert np.abs(tr(st) - s).max() <= 1e-12 * scale


def test_momentum_predictor_is_mirror_symmetric():
    """Mirroring x maps the predicted velocity as a vector field (u_x negated, u_y and u_z
    mirrored), with gravity along z and a pressure that depends on z only."""
    n, h = (13, 11, 9), (1 / 12, 1 / 10, 1 / 8)
    C, U, z = _smooth_state(n, h)
    prm = flow.FlowParams(rho_l=1000.0, rho_g=10.0, mu_l=1e-3, mu_g=1e-4, sigma_t=0.07, g=9.81)
    p = 1000 * 9.81 * (1 - z)
    ut, _ = flow.momentum_predict(C.shape, h, C, U, U, p, 1e-4, prm)
    f = _FLIP[0]
    Um = [-f(U[0]), f(U[1]), f(U[2])]
    utm, _ = flow.momentum_predict(C.shape, h, f(C), Um, Um, f(p), 1e-4, prm)
    back = [-f(utm[0]), f(utm[1]), f(utm[2])]
    for c in range(3):
        assert np.abs(back[c] - ut[c]).max() <= 1e-12 * max(np.abs(a).max() for a in ut), c
