"""Pins of the oracle's explicit flow terms: printed constants, exact quadrature, invariants."""

import os
import sys

import numpy as np
import pytest

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


# ------------------------------------------------ closed-form Petrov-Galerkin coefficient pins
#
# On a separable cubic field C = P(x) + Q(y) + R(z) every coefficient of the compressive scheme
# has a closed form at nodes two or more away from every face, derived here by Taylor expansion
# instead of by applying the assembled filters:
#   * the pointwise gradient m^-1 f(C; w_x) is the central difference (P_{i+1} - P_{i-1}) / 2h_x
#     (the y and z mass factors of w_x = G (x) M (x) M sum to the lumped volume), which for a cubic
#     is P'(x) + p3 h_x^2;
#   * with a uniform velocity, g = u.grad C is quadratic along each axis, and the consistent mass
#     over the lumped mass minus the identity acts on a quadratic as (g_{i-1} + 4 g_i + g_{i+1})/6
#     - g_i = h^2 g'' / 6, so a_C = alpha_a (u p3 h_x^2 + v q3 h_y^2 + w r3 h_z^2), a constant.
# The coefficients that follow are evaluated from these inputs with the printed constants of
# tests/golden/vof_constants.txt, one equation at a time, for three time steps: one that leaves
# every coefficient inside [-k_min, k_max], one that clamps about half of the positive ones at
# k_max and one that clamps about half of the negative ones at -k_min.


def _printed():
    out = {}
    for line in open(os.path.join(GOLDEN, "vof_constants.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def _cubic(c, x0):
    """P(t) = c0 + c1 s + c2 s^2 + c3 s^3 with s = t - x0, and P'(t)."""
    return (lambda t: c[0] + c[1] * (t - x0) + c[2] * (t - x0) ** 2 + c[3] * (t - x0) ** 3,
            lambda t: c[1] + 2 * c[2] * (t - x0) + 3 * c[3] * (t - x0) ** 2)


_VOF_N, _VOF_H = (11, 13, 9), (0.1, 0.05, 0.08)              # anisotropic spacing
_VOF_CUBICS = (((0.45, -0.3, 0.0, 25.0), 0.5),               # P: an extremum inside (S^x < 0)
               ((0.0, 0.9, 1.0, -8.0), 0.3),                 # Q
               ((0.0, 0.4, 0.0, 3.0), 0.32))                 # R
_VOF_VEL = (0.7, -0.4, 0.25)
_INNER = (slice(2, -2),) * 3


def _vof_closed_form(dt):
    """Returns (C, velocity fields, expected parts on the inner nodes) for the separable cubic."""
    K = _printed()
    h = _VOF_H
    X = node_coords(_VOF_N, h)
    fs = [_cubic(*c) for c in _VOF_CUBICS]
    C = sum(fs[d][0](X[d]) for d in range(3))
    # Taylor: central difference of a cubic, and the mixed-mass residual of a quadratic
    grad = [fs[d][1](X[d]) + _VOF_CUBICS[d][0][3] * h[d] ** 2 for d in range(3)]
    a = K["alpha_a"] * sum(_VOF_VEL[d] * _VOF_CUBICS[d][0][3] * h[d] ** 2 for d in range(3))
    a = np.full(C.shape, a)
    # Eq. efficient-kabs (general spacing)
    sabs = sum(np.abs(g) for g in grad)
    k_abs = K["alpha_kabs"] * np.abs(a) * sum(h[d] * np.abs(grad[d]) for d in range(3)) \
        / (K["eps_k"] + sabs * sabs / 3)
    # Eqs. Sx-lin..Sz-lin on nodal values, then the 0.95 / 0.05 override (S = -1)
    S = []
    for d in range(3):
        P = fs[d][0]
        t = X[d]
        raw = (P(t) - P(t - h[d])) * (P(t + h[d]) - P(t))
        S.append(np.where((C > K["detect_hi"]) | (C < K["detect_lo"]), -1.0, raw))
    w_plus = [np.clip(-K["K_plus"] * s, 0.0, 1.0) for s in S]      # -max(-1, min(0, K+ S))
    w_minus = [np.clip(K["K_minus"] * s, 0.0, 1.0) for s in S]     # min(1, max(0, K- S))
    # Eqs. normalisation and negativek
    g2 = sum(g * g for g in grad)
    proj = sum(_VOF_VEL[d] * grad[d] for d in range(3)) / (K["eps_x"] + g2)
    ustar_abs = sum(np.abs(grad[d] * proj) for d in range(3))
    speed2 = sum(v * v for v in _VOF_VEL)
    k_neg = -K["beta"] * speed2 / (K["eps_x"] + g2 * ustar_abs / 3)
    # Eq. positivek, the directional combination, and the clamp of Eq. alpha_min_and_max
    k_lo = K["alpha_min"] * max(h) ** 2 / dt
    k_hi = K["alpha_max"] * min(h) ** 2 / dt
    k = [np.clip(w_plus[d] * K["K_pos"] * k_abs + w_minus[d] * k_neg / h[d], -k_lo, k_hi)
         for d in range(3)]
    vel = [np.full(C.shape, v) for v in _VOF_VEL]
    expect = {"grad": grad, "a_C": a, "k_abs": k_abs, "S": S, "w_plus": w_plus,
              "w_minus": w_minus, "k_neg": k_neg, "k": k}
    return C, vel, {key: ([f[_INNER] for f in val] if isinstance(val, list) else val[_INNER])
                    for key, val in expect.items()}


def _close(got, want, rel=1e-12, floor=1e-300):
    return np.all(np.abs(got - want) <= rel * np.abs(want) + floor)


# dt = 1e-11: no clamp; 0.05: k_max clamps part of the positive side; 3.5e-6: -k_min part of the
# negative side (the spreads are checked in test_closed_form_cases_reach_every_branch)
_VOF_DTS = (1e-11, 0.05, 3.5e-6)


def test_vof_coefficients_match_closed_form():
    """Every intermediate of the compressive Petrov-Galerkin step (Sections 2.3.5-2.3.6) equals
    its closed form on a separable cubic field with anisotropic spacing."""
    for dt in _VOF_DTS:
        C, vel, want = _vof_closed_form(dt)
        _, _, parts = flow.vof_step(C.shape, _VOF_H, C, *vel, dt)
        for key, val in want.items():
            got = parts[key]
            if isinstance(val, list):
                for d in range(3):
                    assert _close(got[d][_INNER], val[d], floor=1e-15 if key == "grad" else 1e-300), (dt, key, d)
            else:
                assert _close(got[_INNER], val), (dt, key)


def test_closed_form_cases_reach_every_branch():
    """The closed-form cases exercise each branch of the scheme at some inner nodes: the detector
    override, S < 0 with a fractional w+, S > 0 with a fractional w-, and both clamps partly
    active, so a slip in any of them changes the pinned values."""
    K = _printed()
    C, _, want = _vof_closed_form(_VOF_DTS[0])
    Ci = C[_INNER]
    assert ((Ci > K["detect_hi"]) | (Ci < K["detect_lo"])).sum() > 10
    assert any(((want["w_plus"][d] > 0) & (want["w_plus"][d] < 1)).sum() > 10 for d in range(3))
    assert any(((want["w_minus"][d] > 0) & (want["w_minus"][d] < 1)).sum() > 10 for d in range(3))
    for i, dt in enumerate(_VOF_DTS):
        _, _, want = _vof_closed_form(dt)
        hi = K["alpha_max"] * min(_VOF_H) ** 2 / dt
        lo = K["alpha_min"] * max(_VOF_H) ** 2 / dt
        at_hi = sum((k == hi).sum() for k in want["k"])
        at_lo = sum((k == -lo).sum() for k in want["k"])
        free_pos = sum(((k > 0) & (k < hi)).sum() for k in want["k"])
        free_neg = sum(((k < 0) & (k > -lo)).sum() for k in want["k"])
        if i == 0:
            assert at_hi == 0 and at_lo == 0 and free_pos > 100 and free_neg > 100
        elif i == 1:
            assert at_hi > 50 and free_pos > 50
        else:
            assert at_lo > 50 and free_neg > 50


def test_vof_update_with_uniform_clamped_diffusion_matches_closed_form():
    """Eqs. Petrov-Cs and transport-indicator-1 in closed form.  C = 0.97 + a separable cubic of
    small amplitude lies in the override band (C > 0.95), so w+ = 1 and w- = 0 in every
    direction; with dt = 10 every 3 k_abs exceeds k_max, so k^d = k_max uniformly.  The
    Petrov-Galerkin term 0.5[D(kC) + k DC - C Dk] is then k_max D_d C, and on a cubic
    D_d C = -m P_d'' (the 1D stiffness row times the y, z masses), while f(C; w_d) = m times the
    central difference P_d' + p3 h_d^2.  So s_C = m [sum_d u_d (P_d' + p3 h_d^2) - k_max sum_d P_d'']
    and C^{n+1} = C - dt s_C / m at nodes two or more from every face."""
    K = _printed()
    n, h, dt = (9, 11, 9), (0.1, 0.05, 0.08), 10.0
    X = node_coords(n, h)
    cub = [(0.002, 0.3, 0.5), (0.001, 0.2, 0.4), (0.0015, 0.1, 0.3)]   # amplitude, c1, c3 about 0.3
    C = 0.97 + sum(A * (c1 * (X[d] - 0.3) + c3 * (X[d] - 0.3) ** 3) for d, (A, c1, c3) in enumerate(cub))
    vel = (0.7, -0.4, 0.25)
    s, Cn, parts = flow.vof_step(C.shape, h, C, *[np.full(C.shape, v) for v in vel], dt)
    k_hi = K["alpha_max"] * min(h) ** 2 / dt
    ring = (slice(1, -1),) * 3
    assert all(np.all(parts["k"][d][ring] == k_hi) for d in range(3))
    m = h[0] * h[1] * h[2]
    d1 = [A * (c1 + 3 * c3 * (X[d] - 0.3) ** 2 + c3 * h[d] ** 2) for d, (A, c1, c3) in enumerate(cub)]
    d2 = [A * 6 * c3 * (X[d] - 0.3) for d, (A, c1, c3) in enumerate(cub)]
    s_want = m * (sum(vel[d] * d1[d] for d in range(3)) - k_hi * sum(d2))
    assert np.abs(s[_INNER] - s_want[_INNER]).max() <= 1e-12 * np.abs(s_want).max()
    assert np.abs(Cn[_INNER] - (C - dt * s_want / m)[_INNER]).max() <= 1e-12


# Momentum (Stage 2): u = P(y) cubic, v and w uniform, uniform C.  For the u component only
# d/dy is non-zero, g = v P~'(y) is quadratic and a = alpha_a v p3 h_y^2; the v and w components
# are uniform, so their a, k_abs and k_square vanish and k_Psi = mu.  The cubic is chosen so that
# k_max, k_abs and k_square are each the smallest of the three at some inner nodes.
_MOM_N, _MOM_H = (9, 17, 9), (0.1, 0.05, 0.08)
_MOM_P3 = 100.0
_MOM_CUBIC = ((0.0, -0.9 * _MOM_P3 * 0.05 ** 2, 0.0, _MOM_P3), 0.4)
_MOM_VW = (0.03, -0.02)
_MOM_C = 0.4


def _momentum_closed_form():
    K = _printed()
    prm = flow.FlowParams()
    h = _MOM_H
    x, y, z = node_coords(_MOM_N, h)
    P, dP = _cubic(*_MOM_CUBIC)
    uh = [P(y), np.full(y.shape, _MOM_VW[0]), np.full(y.shape, _MOM_VW[1])]
    C = np.full(y.shape, _MOM_C)
    rho = prm.rho_l * _MOM_C + prm.rho_g * (1 - _MOM_C)              # Eq. density-n
    mu = prm.mu_l * _MOM_C + prm.mu_g * (1 - _MOM_C)
    py = dP(y) + _MOM_CUBIC[0][3] * h[1] ** 2                        # central difference of a cubic
    a = K["alpha_a"] * _MOM_VW[0] * _MOM_CUBIC[0][3] * h[1] ** 2
    k_max = h[0] * np.abs(uh[0]) + h[1] * abs(_MOM_VW[0]) + h[2] * abs(_MOM_VW[1])   # Eq. max-k
    k_abs = K["alpha_kabs"] * abs(a) * h[1] * np.abs(py) / (K["eps_k"] + py * py / 3)  # efficient-kabs
    h_psi = h[1] * np.abs(py) / (K["eps_k"] + np.abs(py))                               # Eq. h_Psi
    k_sq = K["alpha_ksquare"] * a * a * h_psi / (K["eps_k"] + np.abs(_MOM_VW[0] * py) * py * py / 3)
    k_u = rho * np.minimum(k_max, np.minimum(k_abs, k_sq)) + mu                         # Eq. k_Psi-n
    want = {"a": [np.full(y.shape, a), 0 * y, 0 * y], "k_abs": [k_abs, 0 * y, 0 * y],
            "k_square": [k_sq, 0 * y, 0 * y], "k": [k_u, mu + 0 * y, mu + 0 * y]}
    return C, uh, prm, k_max, {key: [f[_INNER] for f in val] for key, val in want.items()}


def test_momentum_diffusivity_matches_closed_form():
    """k_Psi of Eq. k_Psi-n (with Eqs. a_psi, efficient-kabs, h_Psi, k-square, max-k) for each
    velocity component equals its closed form; rho and mu are not 1 and 0."""
    C, uh, prm, k_max, want = _momentum_closed_form()
    parts = {}
    flow.momentum_predict(C.shape, _MOM_H, C, uh, uh, np.zeros(C.shape), 1e-4, prm, parts=parts)
    assert _close(parts["k_max"][_INNER], k_max[_INNER])
    for key, val in want.items():
        for c in range(3):
            assert _close(parts[key][c][_INNER], val[c], floor=1e-18), (key, c)


def test_momentum_closed_form_reaches_every_branch_of_the_min():
    _, _, _, k_max, want = _momentum_closed_form()
    which = np.argmin(np.stack([k_max[_INNER], want["k_abs"][0], want["k_square"][0]]), axis=0)
    assert all((which == i).sum() >= 10 for i in range(3))


# ------------------------------------------------ the pins catch plausible slips in the oracle

_SLIPS = {
    # Eq. efficient-kabs: the special-case denominator (sum |grad|) instead of its square
    "kabs_denominator": ("/ (prm.eps_k + sum_abs ** 2 / 3.0))", "/ (prm.eps_k + sum_abs / 3.0))"),
    # Eq. positivek: K = 1 instead of 3
    "positive_factor": ("k_plus = prm.K_pos * k_abs", "k_plus = k_abs"),
    # Eq. negativek: the /3 of the denominator dropped
    "negk_third": ("+ np.abs(ustar[2])) / 3.0)", "+ np.abs(ustar[2])))"),
    # k^{d-} = k^- / Delta d: the division dropped
    "negk_spacing": ("k_minus = k_neg / h[d]", "k_minus = k_neg"),
    # Eq. alpha_min_and_max: k_max from the largest spacing
    "kmax_spacing": ("k_max = prm.alpha_max * min(h) ** 2 / dt", "k_max = prm.alpha_max * max(h) ** 2 / dt"),
    # ... and k_min from the smallest
    "kmin_spacing": ("k_min = prm.alpha_min * max(h) ** 2 / dt", "k_min = prm.alpha_min * min(h) ** 2 / dt"),
    # Eq. a_psi: alpha_a = 1
    "alpha_a": ("a_C = prm.alpha_a * (", "a_C = 1.0 * ("),
    # the 0.95 / 0.05 detector override removed, or only its upper half kept
    "override": ("S.append(np.where(over, -1.0, s))", "S.append(s)"),
    "override_lo": ("over = (C > prm.detect_hi) | (C < prm.detect_lo)", "over = (C > prm.detect_hi)"),
    # the weights: w+ with the wrong sign, K- dropped from w-
    "w_plus_sign": ("w_plus = [-np.maximum(", "w_plus = [np.maximum("),
    "w_minus_gain": ("np.maximum(0.0, prm.K_minus * s))", "np.maximum(0.0, s))"),
    # Eq. normalisation without its denominator
    "ustar_norm": ("/ (prm.eps_x + gradsq)\n", "\n"),
    # Eq. k-square with alpha_kabs, or without its /3
    "alpha_ksquare": ("k_sq = (prm.alpha_ksquare * a * a", "k_sq = (prm.alpha_kabs * a * a"),
    "ksq_third": ("* (pd[0] ** 2 + pd[1] ** 2 + pd[2] ** 2) / 3.0))", "* (pd[0] ** 2 + pd[1] ** 2 + pd[2] ** 2)))"),
    # Eq. h_Psi with the squared sum
    "h_psi": ("h_psi = hsum / (prm.eps_k + sab)", "h_psi = hsum / (prm.eps_k + sab ** 2)"),
    # Eq. max-k without the spacings
    "kmax_field": ("kmax = h[0] * np.abs(uh[0]) + h[1] * np.abs(uh[1]) + h[2] * np.abs(uh[2])",
                   "kmax = np.abs(uh[0]) + np.abs(uh[1]) + np.abs(uh[2])"),
    # Eq. Petrov-Cs: the C Dk term with the wrong sign; Eq. transport-indicator-1 without m
    "pg_sign": ("- C * fem.apply_assembled(D, kd[d]))", "+ C * fem.apply_assembled(D, kd[d]))"),
    "update_mass": ("C_next = C - dt * s_C / m", "C_next = C - dt * s_C"),
    # Eq. k_Psi-n: rho dropped, k_abs dropped from the min, mu dropped
    "kpsi_rho": ("k = rho * np.minimum(kmax, np.minimum(k_abs, k_sq)) + mu",
                 "k = np.minimum(kmax, np.minimum(k_abs, k_sq)) + mu"),
    "kpsi_kabs": ("k = rho * np.minimum(kmax, np.minimum(k_abs, k_sq)) + mu",
                  "k = rho * np.minimum(kmax, k_sq) + mu"),
    "kpsi_mu": ("k = rho * np.minimum(kmax, np.minimum(k_abs, k_sq)) + mu",
                "k = rho * np.minimum(kmax, np.minimum(k_abs, k_sq))"),
}


def _mutant(old, new):
    """A copy of oracle.flow with one source substitution (the slip is planted in the oracle, on
    the CPU; the product path is not involved)."""
    import importlib.util
    import types
    src_path = flow.__file__
    src = open(src_path).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._flow_mutant")
    mod.__package__ = "oracle"
    mod.__file__ = src_path
    exec(compile(src.replace(old, new), src_path, "exec"), mod.__dict__)
    assert importlib.util.find_spec("oracle") is not None
    return mod


_PINS = ("test_uniform_field_stays_uniform", "test_mass_conserved_in_divergence_free_wall_tangent_flow",
         "test_vof_update_with_uniform_clamped_diffusion_matches_closed_form", "test_linear_profile_has_no_positive_weight",
         "test_invariant_direction_advection_leaves_interior_unchanged",
         "test_momentum_predictor_advects_a_linear_field_exactly",
         "test_vof_coefficients_match_closed_form", "test_momentum_diffusivity_matches_closed_form")


@pytest.mark.parametrize("slip", sorted(_SLIPS))
def test_pins_catch_planted_mistakes(monkeypatch, slip):
    """Each plausible slip in the coefficient chains, planted in a copy of the oracle, makes at
    least one pin fail."""
    mod = _mutant(*_SLIPS[slip])
    monkeypatch.setattr(sys.modules[__name__], "flow", mod)
    failed = []
    for name in _PINS:
        try:
            globals()[name]()
        except AssertionError:
            failed.append(name)
    assert failed, slip
