"""Pins of the oracle's finite-element filters against printed values and closed forms.

Each test fixes the oracle to something outside itself: a filter printed in the paper, an
exact polynomial identity of Q1 elements, or a worked example.  None re-types the oracle's
formula.
"""

import itertools
import os

import numpy as np
import pytest

from oracle import fem, mg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_slices(name):
    slices, cur = [], None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#") or line.startswith("scale"):
            continue
        if line.startswith("slice"):
            cur = []
            slices.append(cur)
            continue
        cur.append(line.split())
    return slices


def test_wx_equals_printed_filter():
    """Section 2.2.3: w_x = m_l/(72 dx) [..] for linear elements, any (dx, dy, dz)."""
    printed = np.array(_read_slices("wx_linear_filter.txt"), dtype=float)
    for h in [(1.0, 1.0, 1.0), (0.25, 0.5, 2.0), (1 / 32, 1 / 64, 1 / 32)]:
        ml = h[0] * h[1] * h[2]
        ei = fem.element_integrals(h)
        w = fem.interior_filter(ei["grad"][0])
        np.testing.assert_allclose(w, printed * ml / (72 * h[0]), rtol=0, atol=1e-15 * ml / h[0])
        # w_y and w_z are the same filter with the axes exchanged
        wy = fem.interior_filter(ei["grad"][1])
        np.testing.assert_allclose(wy, np.swapaxes(printed, 1, 2) * ml / (72 * h[1]),
                                   atol=1e-15 * ml / h[1])
        wz = fem.interior_filter(ei["grad"][2])
        np.testing.assert_allclose(wz, np.swapaxes(printed, 0, 2) * ml / (72 * h[2]),
                                   atol=1e-15 * ml / h[2])


def test_uniform_laplacian_filter_values():
    """Q1 stiffness on a uniform grid: h*(8/3, 0, -1/6, -1/12) for centre/face/edge/corner."""
    h = 0.37
    w = fem.interior_filter(fem.element_integrals((h, h, h))["stiff"])
    expect = {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        nnz = abs(dx) + abs(dy) + abs(dz)
        assert abs(w[dz + 1, dy + 1, dx + 1] - h * expect[nnz]) < 1e-15


def test_row_sums_vanish_everywhere():
    """The weak Laplacian annihilates constants at every node, boundary rows included."""
    g = mg.Grid((9, 5, 7), (0.3, 0.7, 1.1))
    y = mg.stencil_apply(g, np.ones(g.shape))
    assert np.abs(y).max() < 1e-14


def test_quadratic_field_exact():
    """-lap(x^2+y^2+z^2) = -6 exactly: (A q)_i = -6 m_l at interior nodes (Q1 is exact here)."""
    n, h = (7, 6, 9), (0.2, 0.35, 0.15)
    g = mg.Grid(n, h)
    from synth import node_coords
    x, y, z = node_coords(n, h)
    Aq = mg.stencil_apply(g, x * x + y * y + z * z)
    ml = h[0] * h[1] * h[2]
    np.testing.assert_allclose(Aq[1:-1, 1:-1, 1:-1], -6 * ml, rtol=1e-12)


def test_linear_field_gradient_and_mass():
    """m_l^-1 f(x; w_x) = 1 at interior nodes; sum of w_m = m_l; lumped mass = m_l inside."""
    n, h = (6, 6, 6), (0.2, 0.3, 0.4)
    from synth import node_coords
    x, y, z = node_coords(n, h)
    ei = fem.element_integrals(h)
    ml = h[0] * h[1] * h[2]
    for d, f in enumerate((x, y, z)):
        gx = fem.apply_assembled(ei["grad"][d], f)
        np.testing.assert_allclose(gx[1:-1, 1:-1, 1:-1] / ml, 1.0, rtol=1e-13)
    wm = fem.interior_filter(ei["mass"])
    assert abs(wm.sum() - ml) < 1e-15
    # consistent mass of the tensor product (h/6)[1,4,1] per axis
    one = np.array([1.0, 4.0, 1.0])
    expect = np.einsum("i,j,k->ijk", one * h[2] / 6, one * h[1] / 6, one * h[0] / 6)
    np.testing.assert_allclose(wm, expect, atol=1e-16)
    lm = fem.lumped_mass(n, h)  # shape argument only
    assert abs(lm[2, 2, 2] - ml) < 1e-16
    assert abs(lm[0, 0, 0] - ml / 8) < 1e-16 and abs(lm[0, 2, 2] - ml / 2) < 1e-16


def test_generic_filter_fd_laplacian_and_fig1():
    """Section 2.2.2 filter application reproduces the FD filter and the Fig. 1 example."""
    rng = np.random.default_rng(3)
    dx, dy, dz = 0.5, 0.25, 2.0
    w = np.zeros((3, 3, 3))
    w[1, 1, 1] = 2 / dx**2 + 2 / dy**2 + 2 / dz**2
    w[1, 1, 0] = w[1, 1, 2] = -1 / dx**2
    w[1, 0, 1] = w[1, 2, 1] = -1 / dy**2
    w[0, 1, 1] = w[2, 1, 1] = -1 / dz**2
    # the fixture's layout: slices kk, rows jj, cols ii
    sl = _read_slices("fd_laplacian_filter.txt")
    table = {"0": 0.0, "-1/dz2": -1 / dz**2, "-1/dy2": -1 / dy**2, "-1/dx2": -1 / dx**2,
             "c": 2 / dx**2 + 2 / dy**2 + 2 / dz**2}
    printed = np.array([[[table[v] for v in row] for row in s] for s in sl])
    np.testing.assert_array_equal(printed, w)
    C = rng.standard_normal((6, 7, 8))
    out = fem.filter_apply(C, printed)
    c = C[1:-1, 1:-1, 1:-1]
    ref = ((2 * c - C[1:-1, 1:-1, :-2] - C[1:-1, 1:-1, 2:]) / dx**2
           + (2 * c - C[1:-1, :-2, 1:-1] - C[1:-1, 2:, 1:-1]) / dy**2
           + (2 * c - C[:-2, 1:-1, 1:-1] - C[2:, 1:-1, 1:-1]) / dz**2)
    np.testing.assert_allclose(out, ref, rtol=1e-13)
    # Fig. 1: the 2D filter on a single z-slice, Y33 from the 5x5 image with halo
    f2 = np.loadtxt(os.path.join(GOLDEN, "fig1_fd_example.txt"))
    img = rng.integers(0, 9, size=(7, 7)).astype(float)
    w3 = np.zeros((3, 3, 3))
    w3[1] = f2
    Y = fem.filter_apply(img[None, :, :].repeat(3, axis=0), w3)[0]
    i = j = 3
    assert Y[i - 1, j - 1] == 4 * img[i, j] - (img[i, j - 1] + img[i, j + 1] + img[i - 1, j] + img[i + 1, j])


def test_variable_coefficient_identity_properties():
    """Eq. k-T: symmetric, zero row sums, k = const gives k L, exact on (1+x) * x."""
    rng = np.random.default_rng(0)
    g = mg.Grid((5, 4, 6), (0.3, 0.5, 0.2))
    k = np.exp(rng.standard_normal(g.shape))
    A, _ = mg.dense_matrix(g, k)
    np.testing.assert_allclose(A, A.T, atol=1e-14)
    assert np.abs(A.sum(axis=1)).max() < 1e-13
    np.testing.assert_allclose(np.diag(A), mg.diagonal(g, k).ravel(), rtol=1e-13)
    L, _ = mg.dense_matrix(g)
    A3, _ = mg.dense_matrix(g, np.full(g.shape, 3.0))
    np.testing.assert_allclose(A3, 3 * L, atol=1e-13)
    # -d/dx((1 + x) d/dx x) = -1: exact for Q1 at interior nodes, (A u)_i = -m_l
    from synth import node_coords
    n, h = (7, 7, 7), (0.1, 0.2, 0.3)
    gg = mg.Grid(n, h)
    x, _, _ = node_coords(n, h)
    Au = mg.stencil_apply(gg, x, 1.0 + x)
    np.testing.assert_allclose(Au[1:-1, 1:-1, 1:-1], -h[0] * h[1] * h[2], rtol=1e-12)


def test_galerkin_identity():
    """P^T A_h P = A_2h on the free nodes (Dirichlet and natural faces); pins R, P and A."""
    cases = [((9, 9, 9), (True,) * 6), ((9, 9, 9), (False,) * 6),
             ((9, 5, 17), (False, False, True, False, False, True))]
    for n, bc in cases:
        g = mg.Grid(n, (0.125, 0.3, 0.07), bc)
        gc = g.coarse()
        Af, ff = mg.dense_matrix(g)
        Ac, fc = mg.dense_matrix(gc)
        # dense P on free nodes: columns = prolongation of coarse unit vectors
        P = np.zeros((ff.size, fc.size))
        for c, j in enumerate(fc):
            e = np.zeros(gc.shape)
            e.ravel()[j] = 1.0
            P[:, c] = mg.prolong(g, e).ravel()[ff]
        np.testing.assert_allclose(P.T @ Af @ P, Ac, atol=1e-13 * np.abs(Ac).max())
        # restriction is the transpose of prolongation (after masking)
        R = np.zeros((fc.size, ff.size))
        for c, j in enumerate(ff):
            e = np.zeros(g.shape)
            e.ravel()[j] = 1.0
            R[:, c] = mg.restrict(g, e).ravel()[fc]
        np.testing.assert_allclose(R, P.T, atol=0)


@pytest.mark.parametrize("planted", ["grad_transposed", "drop_z_stiffness", "mass_weight"])
def test_pins_catch_planted_mistakes(monkeypatch, planted):
    """A plausible slip in the element integrals makes at least one pin above fail."""
    real = fem.element_integrals

    def broken(h):
        ei = real(h)
        ei = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in ei.items()}
        if planted == "grad_transposed":
            ei["grad"] = np.transpose(ei["grad"], (0, 2, 1)).copy()
        elif planted == "drop_z_stiffness":
            ei["stiff"] = ei["dd"][0] + ei["dd"][1]
        elif planted == "mass_weight":
            ei["mass"] = ei["mass"] * 1.01
        return ei

    monkeypatch.setattr(fem, "element_integrals", broken)
    failures = 0
    for t in (test_wx_equals_printed_filter, test_uniform_laplacian_filter_values,
              test_quadratic_field_exact, test_linear_field_gradient_and_mass):
        try:
            t()
        except AssertionError:
            failures += 1
    assert failures >= 1
