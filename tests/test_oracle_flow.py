"""Pins of the oracle's explicit flow terms: printed constants, exact quadrature, invariants."""

import os

import numpy as np

from oracle import fem, flow
from synth import node_coords

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
