"""Pressure-correction multigrid of the paper, written out plainly in FP64 (ORACLE, test use only).

The paper solves both pressure equations (Stage 1, Eq. ph_disc; Stage 3, Eq. ph_disc2) with a
sawtooth multigrid cycle built as a U-Net (Section 2.4 and the multigrid figure), with Jacobi
smoothing (Section 1.1).  The figure is not available and the text does not fix restriction,
prolongation, sweep counts or the coarsest solve, so this module takes the following reading:

* vertex grids with n = 2^k + 1 nodes per axis (any odd n >= 5 coarsens); coarse node I sits at
  fine node 2I; coarsening stops when an axis has 3 nodes or an even count;
* prolongation P = trilinear interpolation, restriction R = P^T (unscaled);
* coarse operators are Galerkin, A_{l+1} = P^T A_l P on the free nodes.  For a constant
  coefficient this equals the operator rediscretised at spacing 2^l h, which is what is used
  then (the identity is pinned by the tests); for a coefficient field the triple product is
  formed explicitly (a rediscretised operator with an averaged coefficient makes the cycle
  diverge at a 1000:1 density ratio);
* one sawtooth V(0,1) cycle: residual on the finest level, restriction to the coarsest level,
  exact coarsest solve, then on the way up prolongation followed by one weighted-Jacobi sweep
  (omega = 2/3) on every level, the finest level included;
* Dirichlet nodes (the paper fixes the halo to the prescribed value there, Section 2.3.3) are stored in the
  array and never change; their residual and correction are zero.  Zero-derivative faces use
  natural FE truncation (the boundary row of the assembled operator).

The operator A is the SPD weak form of -laplacian (positive diagonal), see the sign discussion
of Eq. ph_disc; with a coefficient field k it is the paper's Eq. k-T,
A_k x = 1/2 [ L(k x) + k L x - x L k ].
"""

from dataclasses import dataclass

import numpy as np

from . import fem


@dataclass(frozen=True)
class Grid:
    """Vertex grid: ``n`` = (nx, ny, nz) nodes, spacing ``h``, Dirichlet flag per face.

    ``dirichlet`` = (x-, x+, y-, y+, z-, z+); a face that is not Dirichlet is natural.
    """
    n: tuple
    h: tuple
    dirichlet: tuple = (False,) * 6

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def coarse(self):
        return Grid(tuple((m + 1) // 2 for m in self.n), tuple(2.0 * v for v in self.h),
                    self.dirichlet)

    def can_coarsen(self):
        return all(m >= 5 and m % 2 == 1 for m in self.n)


def dirichlet_mask(g):
    """True at nodes that lie on a Dirichlet face."""
    m = np.zeros(g.shape, dtype=bool)
    dx0, dx1, dy0, dy1, dz0, dz1 = g.dirichlet
    if dx0:
        m[:, :, 0] = True
    if dx1:
        m[:, :, -1] = True
    if dy0:
        m[:, 0, :] = True
    if dy1:
        m[:, -1, :] = True
    if dz0:
        m[0, :, :] = True
    if dz1:
        m[-1, :, :] = True
    return m


def is_singular(g):
    """All faces natural: A has the constants as its null space."""
    return not any(g.dirichlet)


def hierarchy(g):
    """Grids from fine (level 0) to coarsest, per the coarsening rule above."""
    out = [g]
    while out[-1].can_coarsen():
        out.append(out[-1].coarse())
    return out


# ---------------------------------------------------------------- operators (Section 2.2.4)

def _L(g, x):
    """Constant-coefficient weak -laplacian (the paper's w_lap filter, assembled)."""
    return fem.apply_assembled(fem.element_integrals(g.h)["stiff"], x)


def stencil_apply(g, x, k=None):
    """y = A x; with a coefficient field k, the identity of Eq. k-T (Section 2.2.4)."""
    x = np.asarray(x, dtype=np.float64)
    if k is None:
        return _L(g, x)
    return 0.5 * (_L(g, k * x) + k * _L(g, x) - x * _L(g, k))


def diagonal(g, k=None):
    """Diagonal of A: L_ii, or L_ii k_i - 1/2 (L k)_i for Eq. k-T."""
    d = fem.assembled_diagonal(fem.element_integrals(g.h)["stiff"], g.shape)
    if k is None:
        return d
    return d * k - 0.5 * _L(g, k)


def residual(g, b, x, k=None):
    """r = b - A x at free nodes, 0 at Dirichlet nodes."""
    r = b - stencil_apply(g, x, k)
    r[dirichlet_mask(g)] = 0.0
    return r


def jacobi(g, b, x, k=None, omega=2.0 / 3.0):
    """One weighted-Jacobi sweep x <- x + omega D^-1 (b - A x); Dirichlet nodes unchanged."""
    return x + omega * residual(g, b, x, k) / diagonal(g, k)


# ---------------------------------------------------------------- inter-grid transfers

def prolong_1d(nc):
    """(2 nc - 1) x nc linear interpolation: injection at even fine nodes, average at odd."""
    nf = 2 * nc - 1
    P = np.zeros((nf, nc))
    for I in range(nc):
        P[2 * I, I] = 1.0
    for I in range(nc - 1):
        P[2 * I + 1, I] = 0.5
        P[2 * I + 1, I + 1] = 0.5
    return P


def _along(M, a, axis):
    return np.moveaxis(np.tensordot(M, a, axes=([1], [axis])), 0, axis)


def prolong_raw(gc, ec):
    """Trilinear interpolation of a coarse field onto the fine grid (no boundary masking)."""
    nx, ny, nz = gc.n
    e = _along(prolong_1d(nz), ec, 0)
    e = _along(prolong_1d(ny), e, 1)
    return _along(prolong_1d(nx), e, 2)


def restrict_raw(gf, rf):
    """R = P^T applied to a fine field (weights prod_d (1/2)^|offset_d|; no masking)."""
    nx, ny, nz = gf.coarse().n
    r = _along(prolong_1d(nz).T, rf, 0)
    r = _along(prolong_1d(ny).T, r, 1)
    return _along(prolong_1d(nx).T, r, 2)


def prolong(gf, ec):
    """e_f = P e_c with e_f = 0 at fine Dirichlet nodes."""
    e = prolong_raw(gf.coarse(), ec)
    e[dirichlet_mask(gf)] = 0.0
    return e


def restrict(gf, rf):
    """r_c = R r_f with r_c = 0 at coarse Dirichlet nodes."""
    r = restrict_raw(gf, rf)
    r[dirichlet_mask(gf.coarse())] = 0.0
    return r


# ---------------------------------------------------------------- coarsest solve

def dense_matrix(g, k=None):
    """The operator on the free nodes as a dense matrix (columns = A applied to unit vectors)."""
    free = np.flatnonzero(~dirichlet_mask(g).ravel())
    A = np.zeros((free.size, free.size))
    for c, j in enumerate(free):
        e = np.zeros(g.shape)
        e.ravel()[j] = 1.0
        A[:, c] = stencil_apply(g, e, k).ravel()[free]
    return A, free


def coarse_solve(g, r, k=None):
    """Exact solve A e = r on the coarsest grid; minimum-norm (zero-mean) when singular."""
    A, free = dense_matrix(g, k)
    rhs = r.ravel()[free]
    sol = min_norm_solve(A, rhs) if is_singular(g) else np.linalg.solve(A, rhs)
    e = np.zeros(int(np.prod(g.shape)))
    e[free] = sol
    return e.reshape(g.shape)


def min_norm_solve(A, rhs):
    """Minimum-norm solution of a singular symmetric system (null space: the constants).

    Eigen-decomposition with a numerical-rank cutoff of 1e-10 relative to the largest
    eigenvalue: the exact null eigenvalue is computed at rounding level, and an SVD cutoff at
    machine precision would keep it and add a large spurious constant.
    """
    w, V = np.linalg.eigh(0.5 * (A + A.T))
    keep = np.abs(w) > 1e-10 * np.abs(w).max()
    return V[:, keep] @ ((V[:, keep].T @ rhs) / w[keep])


# ---------------------------------------------------------------- cycle and solve

def sparse_laplacian(g):
    """The assembled constant-coefficient operator L as a sparse matrix (element by element)."""
    import scipy.sparse as sp
    Ae = fem.element_integrals(g.h)["stiff"]
    nz, ny, nx = g.shape
    idx = np.arange(nx * ny * nz).reshape(g.shape)
    rows, cols, vals = [], [], []
    for a in range(8):
        ia = idx[fem._elem_slice(g.shape, fem.LOCAL[a])].ravel()
        for b in range(8):
            ib = idx[fem._elem_slice(g.shape, fem.LOCAL[b])].ravel()
            rows.append(ia)
            cols.append(ib)
            vals.append(np.full(ia.size, Ae[a, b]))
    n = nx * ny * nz
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def sparse_operator(g, k=None):
    """A as a sparse matrix; with k, Eq. k-T as matrices: 1/2 (diag(k) L + L diag(k)) - 1/2 diag(L k)."""
    import scipy.sparse as sp
    L = sparse_laplacian(g)
    if k is None:
        return L
    kv = np.asarray(k, dtype=np.float64).ravel()
    Dk = sp.diags(kv)
    return (0.5 * (Dk @ L + L @ Dk) - 0.5 * sp.diags(L @ kv)).tocsr()


def sparse_prolongation(gf):
    """P as a sparse matrix: the tensor product of the 1D interpolations, restricted so that
    fine Dirichlet rows and coarse Dirichlet columns are zero."""
    import scipy.sparse as sp
    gc = gf.coarse()
    P = sp.kron(sp.kron(sp.csr_matrix(prolong_1d(gc.n[2])), sp.csr_matrix(prolong_1d(gc.n[1]))),
                sp.csr_matrix(prolong_1d(gc.n[0]))).tocsr()
    keep_f = sp.diags((~dirichlet_mask(gf)).ravel().astype(np.float64))
    keep_c = sp.diags((~dirichlet_mask(gc)).ravel().astype(np.float64))
    return (keep_f @ P @ keep_c).tocsr()


def free_block(g, A):
    """A with the rows and columns of Dirichlet nodes removed (set to zero)."""
    import scipy.sparse as sp
    keep = sp.diags((~dirichlet_mask(g)).ravel().astype(np.float64))
    return (keep @ A @ keep).tocsr()


class Levels:
    """Grid hierarchy and the operator on every level.

    Level 0 is applied matrix-free (it also acts on stored Dirichlet values).  Coarse levels act
    on corrections that vanish at Dirichlet nodes: with no coefficient field they are the
    rediscretised operators; with a field k they are the Galerkin products P^T A P of the free
    blocks, kept as sparse matrices.
    """

    def __init__(self, g, k=None, omega=2.0 / 3.0):
        self.grids = hierarchy(g)
        self.omega = omega
        self.k = np.asarray(k, dtype=np.float64) if k is not None else None
        self.A = [None] * len(self.grids)
        if self.k is not None:
            A = free_block(g, sparse_operator(g, self.k))
            for l in range(len(self.grids) - 1):
                P = sparse_prolongation(self.grids[l])
                A = (P.T @ A @ P).tocsr()
                self.A[l + 1] = A

    def __len__(self):
        return len(self.grids)

    def apply(self, l, x):
        if l == 0 or self.A[l] is None:
            return stencil_apply(self.grids[l], x, self.k if l == 0 else None)
        return (self.A[l] @ x.ravel()).reshape(x.shape)

    def diag(self, l):
        if l == 0 or self.A[l] is None:
            return diagonal(self.grids[l], self.k if l == 0 else None)
        d = self.A[l].diagonal().reshape(self.grids[l].shape).copy()
        d[dirichlet_mask(self.grids[l])] = 1.0
        return d

    def residual(self, l, b, x):
        r = b - self.apply(l, x)
        r[dirichlet_mask(self.grids[l])] = 0.0
        return r

    def jacobi(self, l, b, x):
        return x + self.omega * self.residual(l, b, x) / self.diag(l)

    def coarse_solve(self, r):
        l = len(self.grids) - 1
        g = self.grids[l]
        if l == 0 or self.A[l] is None:
            return coarse_solve(g, r, self.k if l == 0 else None)
        free = np.flatnonzero(~dirichlet_mask(g).ravel())
        A = self.A[l].toarray()[np.ix_(free, free)]
        rhs = r.ravel()[free]
        sol = min_norm_solve(A, rhs) if is_singular(g) else np.linalg.solve(A, rhs)
        e = np.zeros(int(np.prod(g.shape)))
        e[free] = sol
        return e.reshape(g.shape)


def vcycle(lv, x, b):
    """One sawtooth V(0,1) cycle (reading of the multigrid figure of Section 2.4).

    down: r_0 = b - A_0 x, r_{l+1} = R r_l;  coarsest: e_L = A_L^-1 r_L;
    up:   e_l = P e_{l+1} then one Jacobi sweep on A_l e_l = r_l (l = L-1 .. 1);
    finest: x <- x + P e_1 then one Jacobi sweep on A_0 x = b.
    """
    G = lv.grids
    L = len(G) - 1
    r = [lv.residual(0, b, x)]
    if L == 0:
        return x + lv.coarse_solve(r[0])
    for l in range(L):
        r.append(restrict(G[l], r[l]))
    e = lv.coarse_solve(r[L])
    for l in range(L - 1, 0, -1):
        e = prolong(G[l], e)
        e = lv.jacobi(l, r[l], e)
    x = x + prolong(G[0], e)
    return lv.jacobi(0, b, x)


def rel_residual(g, b, x, k=None):
    """||b - A x||_2 / ||b||_2 over the free nodes."""
    return float(np.linalg.norm(residual(g, b, x, k)) / np.linalg.norm(np.where(dirichlet_mask(g), 0.0, b)))


def pressure_solve(g, b, x0=None, k=None, rtol=1e-8, max_cycles=100, omega=2.0 / 3.0,
                   fixed_cycles=None):
    """Repeat V-cycles from x0 (default 0) until ||b - A x|| / ||b|| <= rtol.

    With ``fixed_cycles`` the paper's fixed count (20 per pressure solve, Section 2.4 Stage 1)
    is run regardless of rtol.  Returns (x, history) with history[c] the relative residual
    after c cycles (history[0] for x0).
    """
    lv = Levels(g, k, omega)
    x = np.zeros(g.shape) if x0 is None else np.array(x0, dtype=np.float64)
    hist = [rel_residual(g, b, x, k)]
    ncyc = fixed_cycles if fixed_cycles is not None else max_cycles
    for _ in range(ncyc):
        if fixed_cycles is None and hist[-1] <= rtol:
            break
        x = vcycle(lv, x, b)
        hist.append(rel_residual(g, b, x, k))
    return x, hist


def mass_weighted_mean(g, x):
    """sum m_i x_i / sum m_i with m the lumped nodal volume (to compare singular solutions)."""
    m = fem.lumped_mass(g.shape, g.h)
    return float((m * x).sum() / m.sum())


def pressure_solve_fcg(g, b, x0=None, k=None, rtol=1e-8, max_iters=200, inner_cycles=1,
                       omega=2.0 / 3.0):
    """Flexible conjugate gradients (Notay, SIAM J. Sci. Comput. 22, 2000), truncated to one
    previous direction, preconditioned by ``inner_cycles`` V-cycles on A z = r from z = 0.

    Not in the paper: the paper repeats cycles (Section 2.4); this outer loop is what makes the
    variable-coefficient pressure solve at a 1000:1 density ratio converge in few cycles.
    Recurrences per iteration:  z = B r;  p = z - (z.q_old)/(p_old.q_old) p_old;  q = A p;
    alpha = (p.r)/(p.q);  x += alpha p;  r -= alpha q.  Returns (x, history) with the relative
    norm of the recurrence residual after every iteration (history[0] for x0).
    """
    lv = Levels(g, k, omega)
    mask = dirichlet_mask(g)
    bm = np.where(mask, 0.0, b)
    nb = np.linalg.norm(bm)
    x = np.zeros(g.shape) if x0 is None else np.array(x0, dtype=np.float64)
    r = lv.residual(0, b, x)
    hist = [float(np.linalg.norm(r) / nb)]
    p_old = q_old = None
    for _ in range(max_iters):
        if hist[-1] <= rtol:
            break
        z = np.zeros(g.shape)
        for _ in range(inner_cycles):
            z = vcycle(lv, z, r)
        p = z
        if p_old is not None:
            p = z - (float((z * q_old).sum()) / float((p_old * q_old).sum())) * p_old
        q = stencil_apply(g, p, lv.k)
        q[mask] = 0.0
        alpha = float((p * r).sum()) / float((p * q).sum())
        x = x + alpha * p
        r = r - alpha * q
        p_old, q_old = p, q
        hist.append(float(np.linalg.norm(r) / nb))
    return x, hist
