"""GPU parity of the single multigrid steps (C ABI via the binding) against the FP64 oracle.

Element-by-element comparison on seeded inputs, on grids that span several 32 x 16 tiles and
several z-chunks, with ragged edges, every face condition mix, all three storage types, and
with and without a coefficient field.  Tolerance: |gpu - oracle| <= tol * sum_j |A_ij x_j|
(+ tol * |value| for the final rounding), tol = 1e-13 (FP64), 4e-6 (FP32 accumulate), 1.2e-2
(BF16 storage: 2^-8 rounding of the stored output plus FP32 accumulation).
"""

import numpy as np
import pytest
import torch

from oracle import fem, mg
from tests.gpu_util import TDT, TOL, abs_bound, need_gpu, ogrid, rounded, seeded

pytestmark = pytest.mark.gpu

GRIDS = [
    ((33, 33, 33), (1 / 32,) * 3, (True,) * 6),
    ((37, 21, 19), (0.05, 0.1, 0.07), (False,) * 6),
    ((65, 17, 9), (1 / 64, 1 / 16, 1 / 8), (False, False, True, False, False, True)),
    ((5, 3, 3), (0.25, 0.5, 0.5), (False,) * 5 + (True,)),
    ((129, 65, 65), (1 / 32, 1 / 64, 1 / 32), (False,) * 5 + (True,)),
]


def _setup(n, h, bc, dt, vc, seed=0):
    from paper_2401_06755_gb300 import nn4
    g = ogrid(n, h, bc)
    G = nn4.Grid(n, h, tuple(nn4.DIRICHLET if d else nn4.NATURAL for d in bc))
    x = rounded(seeded(g.shape, seed), dt)
    b = rounded(seeded(g.shape, seed + 1) * np.prod(h), dt)
    k = rounded(np.exp(0.5 * seeded(g.shape, seed + 2)), dt) if vc else None
    T = TDT[dt]
    dev = lambda a: nn4.to_field(a, G, T) if a is not None else None
    return nn4, g, G, x, b, k, dev(x), dev(b), dev(k)


def _cmp(got, ref, bound, dt):
    tol = TOL[dt]
    err = np.abs(got - ref)
    lim = tol * (bound + np.abs(ref)) + 1e-300
    bad = err > lim
    assert not bad.any(), f"{bad.sum()} of {bad.size} outside tolerance; worst ratio {np.max(err / lim):.3g}"


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("vc", [False, True])
@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_stencil_apply_residual_jacobi(gi, vc, dt):
    need_gpu()
    n, h, bc = GRIDS[gi]
    nn4, g, G, x, b, k, X, B, K = _setup(n, h, bc, dt, vc, seed=10 * gi)
    bound = abs_bound(g, x, k)
    y = nn4.nodes(nn4.stencil_apply(G, X, K), G).double().cpu().numpy()
    _cmp(y, mg.stencil_apply(g, x, k), bound, dt)

    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = nn4.nodes(nn4.residual(G, B, X, K, norm2=norm), G).double().cpu().numpy()
    rref = mg.residual(g, b, x, k)
    _cmp(r, rref, bound + np.abs(b), dt)
    nr = float(norm.item())
    # the norm is accumulated in FP64 from the values before storage rounding
    assert abs(nr - (r * r).sum()) <= 3 * TOL[dt] * (r * r).sum() + 1e-300

    xo = nn4.nodes(nn4.jacobi_smooth(G, B, X, K, omega=2 / 3), G).double().cpu().numpy()
    xref = mg.jacobi(g, b, x, k, 2 / 3)
    D = np.abs(mg.diagonal(g, k))
    _cmp(xo, xref, np.abs(x) + (2 / 3) * (bound + np.abs(b)) / D, dt)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("gi", [0, 1, 2, 4])
def test_restrict_prolong(gi, dt):
    need_gpu()
    n, h, bc = GRIDS[gi]
    nn4, g, G, x, b, k, X, B, K = _setup(n, h, bc, dt, False, seed=3 + gi)
    gc = g.coarse()
    rc = nn4.nodes(nn4.restrict(G, X), G.coarse()).double().cpu().numpy()
    ref = mg.restrict(g, x)
    bnd = mg.restrict_raw(g, np.abs(x))
    _cmp(rc, ref, bnd, dt)

    ec = rounded(seeded(gc.shape, 77 + gi), dt)
    EC = nn4.to_field(ec, G.coarse(), TDT[dt])
    ef = nn4.nodes(nn4.prolong(G, EC), G).double().cpu().numpy()
    _cmp(ef, mg.prolong(g, ec), mg.prolong_raw(gc, np.abs(ec)), dt)
    # accumulate onto an existing fine field; Dirichlet nodes stay unchanged
    base = nn4.to_field(x, G, TDT[dt])
    ef2 = nn4.nodes(nn4.prolong(G, EC, base, accumulate=True), G).double().cpu().numpy()
    ref2 = x + mg.prolong(g, ec)
    _cmp(ef2, ref2, np.abs(x) + mg.prolong_raw(gc, np.abs(ec)), dt)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("vc", [False, True])
@pytest.mark.parametrize("gi", [0, 1, 2, 3, 4])
def test_residual_restrict_fused(gi, vc, dt):
    """R (b - A x) in one pass against the oracle's restriction of its residual, element by element
    on the coarse grid (several tiles and z-chunks, ragged in every axis, every face mix), and the
    fine residual's squared norm against the oracle's."""
    need_gpu()
    n, h, bc = GRIDS[gi]
    nn4, g, G, x, b, k, X, B, K = _setup(n, h, bc, dt, vc, seed=20 + gi)
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = nn4.nodes(nn4.residual_restrict(G, B, X, K, norm2=norm), G.coarse()).double().cpu().numpy()
    rf = mg.residual(g, b, x, k)
    ebound = abs_bound(g, x, k) + np.abs(b)  # per fine node: the residual's rounding scale
    _cmp(rc, mg.restrict(g, rf), mg.restrict_raw(g, ebound), dt)
    # the fine residual is not rounded to the storage type here: FP32 (FP64) arithmetic only, then
    # FP32 partial sums along each thread's z-march
    tol = TOL["f32"] if dt != "f64" else TOL["f64"]
    nref = float((rf * rf).sum())
    lim = 2 * tol * float((np.abs(rf) * ebound).sum()) + 3 * tol * nref + 1e-300
    assert abs(norm.item() - nref) <= lim, (norm.item(), nref)


def test_full_size_residual_restrict_sampled():
    """257^3 FP32 residual + restriction with a coefficient field, checked at sampled coarse nodes
    against the oracle's residual on a 7^3 window around each sample, restricted by hand."""
    need_gpu()
    from paper_2401_06755_gb300 import nn4
    n = 257
    h = 1.0 / 256
    G = nn4.Grid((n,) * 3, (h,) * 3)
    rng = np.random.default_rng(6)
    shape = (n, n, n)
    x = rounded(rng.standard_normal(shape), "f32")
    k = rounded(np.exp(rng.standard_normal(shape)), "f32")
    b = rounded(rng.standard_normal(shape) * h ** 3, "f32")
    dev = lambda a: nn4.to_field(a, G, torch.float32)
    rc = nn4.nodes(nn4.residual_restrict(G, dev(b), dev(x), dev(k)), G.coarse()).double().cpu().numpy()
    nc = (n + 1) // 2
    pts = [(0, 0, 0), (128, 128, 128), (64, 0, 127), (15, 7, 17), (14, 6, 16), (0, 100, 8)] + \
        [tuple(int(v) for v in rng.integers(0, nc, 3)) for _ in range(30)]
    w1 = {-1: 0.5, 0: 1.0, 1: 0.5}
    for (I, J, Kc) in pts:
        c = (2 * Kc, 2 * J, 2 * I)
        # fine residuals at c + {-1, 0, 1}^3 are exact on a window reaching two nodes past them
        lo = [max(0, v - 3) for v in c]
        hi = [min(n, v + 4) for v in c]
        sl = tuple(slice(a, b_) for a, b_ in zip(lo, hi))
        sub = mg.Grid(tuple(hi[2 - d] - lo[2 - d] for d in range(3)), (h,) * 3)
        rs = mg.residual(sub, b[sl], x[sl], k[sl])
        es = abs_bound(sub, x[sl], k[sl]) + np.abs(b[sl])
        val = bnd = 0.0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    f = (c[0] + dz, c[1] + dy, c[2] + dx)
                    if not all(0 <= f[d] < n for d in range(3)):
                        continue
                    wgt = w1[dz] * w1[dy] * w1[dx]
                    li = tuple(f[d] - lo[d] for d in range(3))
                    val += wgt * rs[li]
                    bnd += wgt * es[li]
        assert abs(rc[Kc, J, I] - val) <= TOL["f32"] * (bnd + abs(val)), (I, J, Kc)


def test_full_size_stencil_sampled():
    """257^3 FP32 stencil apply with a coefficient field (the timed size), checked at sampled
    nodes against the oracle evaluated on a small neighbourhood of each sample."""
    need_gpu()
    from paper_2401_06755_gb300 import nn4
    n = 257
    h = 1.0 / 256
    g = ogrid((n,) * 3, (h,) * 3, (False,) * 6)
    G = nn4.Grid((n,) * 3, (h,) * 3)
    rng = np.random.default_rng(5)
    x = rounded(rng.standard_normal(g.shape), "f32")
    k = rounded(np.exp(rng.standard_normal(g.shape)), "f32")
    y = nn4.nodes(nn4.stencil_apply(G, nn4.to_field(x, G, torch.float32), nn4.to_field(k, G, torch.float32)), G)
    y = y.double().cpu().numpy()
    pts = [(0, 0, 0), (256, 256, 256), (128, 5, 255), (31, 32, 33), (0, 200, 17)] + \
        [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(40)]
    for (i, j, kk) in pts:
        # a 5^3 window (clipped at the boundary) reproduces the row exactly when the window's
        # own boundary is the domain boundary or two nodes away from the node
        lo = [max(0, c - 2) for c in (kk, j, i)]
        hi = [min(n, c + 3) for c in (kk, j, i)]
        sl = tuple(slice(a, b_) for a, b_ in zip(lo, hi))
        sub = mg.Grid((hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]), (h,) * 3)
        ys = mg.stencil_apply(sub, x[sl], k[sl])
        c = (kk - lo[0], j - lo[1], i - lo[2])
        bnd = abs_bound(sub, x[sl], k[sl])[c]
        assert abs(y[kk, j, i] - ys[c]) <= 4e-6 * (bnd + abs(ys[c])), (i, j, kk)
