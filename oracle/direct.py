"""Exact solutions of the pressure system A x = b (ORACLE, test use only).

The paper states that its network gives the answer of the discretised equations to within the
solver tolerance (Sections 1.1 and 1.2).  So the reference solution of a pressure solve is the
solution of the linear system itself, independent of every multigrid choice: a dense direct
solve on small grids and plain conjugate gradients (Hestenes and Stiefel) on larger ones.
"""

import numpy as np

from . import mg


def solve_dense(g, b, k=None):
    """Dense LU solve on the free nodes; minimum-norm (zero-mean) solution when singular."""
    A, free = mg.dense_matrix(g, k)
    rhs = b.ravel()[free]
    if mg.is_singular(g):
        sol = mg.min_norm_solve(A, rhs)
    else:
        sol = np.linalg.solve(A, rhs)
    x = np.zeros(int(np.prod(g.shape)))
    x[free] = sol
    return x.reshape(g.shape)


def solve_cg(g, b, k=None, rtol=1e-14, max_iter=100000):
    """Unpreconditioned CG on the free nodes from x = 0 until ||r|| <= rtol ||b||.

    For the singular all-natural case the right-hand side must sum to zero; the iterates then
    stay in the range of A and the result is shifted to zero plain mean.
    """
    mask = mg.dirichlet_mask(g)
    b = np.where(mask, 0.0, b)
    x = np.zeros(g.shape)
    r = b.copy()
    p = r.copy()
    rr = float((r * r).sum())
    stop = (rtol * np.linalg.norm(b)) ** 2
    for _ in range(max_iter):
        if rr <= stop:
            break
        Ap = mg.stencil_apply(g, p, k)
        Ap[mask] = 0.0
        alpha = rr / float((p * Ap).sum())
        x += alpha * p
        r -= alpha * Ap
        rr_new = float((r * r).sum())
        p = r + (rr_new / rr) * p
        rr = rr_new
    if mg.is_singular(g):
        x -= x.mean()
    return x
