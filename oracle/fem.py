"""Q1 finite-element integrals and matrix-free assembled operators (ORACLE, test use only).

Section 2.2.3 defines filter weights as integrals of products of basis functions and their
derivatives, built the standard finite-element way; Section 2.2.4 uses the same construction for the second
derivative (Laplacian) filter.  Here the integrals are taken element by element with 2-point
Gauss quadrature per axis (exact for the bilinear-per-axis integrands of Q1), and a global
operator is applied by summing element contributions, which is what assembly means.  Near the
domain boundary a node simply has fewer elements around it (a natural boundary: no boundary term is added).

Arrays are indexed [z, y, x] (x fastest).  Local element node a = ax + 2*ay + 4*az.
"""

import itertools

import numpy as np

_GP = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # Gauss points on [0, 1]
_GW = (0.5, 0.5)                                              # weights on [0, 1]
LOCAL = [(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]   # (ax, ay, az)


def _basis(xi):
    """Trilinear basis N_a(xi) and reference derivatives dN_a/dxi_d at xi in [0,1]^3."""
    N = np.empty(8)
    dN = np.empty((8, 3))
    for a, off in enumerate(LOCAL):
        f = [xi[d] if off[d] else 1.0 - xi[d] for d in range(3)]
        s = [1.0 if off[d] else -1.0 for d in range(3)]
        N[a] = f[0] * f[1] * f[2]
        dN[a, 0] = s[0] * f[1] * f[2]
        dN[a, 1] = f[0] * s[1] * f[2]
        dN[a, 2] = f[0] * f[1] * s[2]
    return N, dN


def element_integrals(h):
    """Element matrices of one hexahedron with edges h = (hx, hy, hz).

    Returns a dict with
      mass[a,b]    = int N_a N_b                       (consistent mass, filter w_m)
      grad[d][a,b] = int N_a dN_b/dx_d                 (first derivative filters w_x, w_y, w_z;
                                                        Section 2.2.3, row = test function a)
      dd[d][a,b]   = int dN_a/dx_d dN_b/dx_d           (directional second derivative filters
                                                        w_xx^PG, w_yy^PG, w_zz^PG; Section 2.2.4)
      stiff[a,b]   = sum_d dd[d][a,b]                  (isotropic diffusion filter w_lap,
                                                        the weak form of -laplacian)
      lumped[a]    = int N_a                           (row sums of mass; lumped mass)
    """
    h = np.asarray(h, dtype=np.float64)
    vol = float(h[0] * h[1] * h[2])
    mass = np.zeros((8, 8))
    grad = np.zeros((3, 8, 8))
    dd = np.zeros((3, 8, 8))
    lumped = np.zeros(8)
    for (i, gx), (j, gy), (k, gz) in itertools.product(enumerate(_GP), repeat=3):
        w = _GW[i] * _GW[j] * _GW[k] * vol
        N, dN = _basis((gx, gy, gz))
        dNdx = dN / h[None, :]
        mass += w * np.outer(N, N)
        lumped += w * N
        for d in range(3):
            grad[d] += w * np.outer(N, dNdx[:, d])
            dd[d] += w * np.outer(dNdx[:, d], dNdx[:, d])
    return {"mass": mass, "grad": grad, "dd": dd, "stiff": dd.sum(axis=0), "lumped": lumped}


def _elem_slice(shape, off):
    nz, ny, nx = shape
    return (slice(off[2], off[2] + nz - 1), slice(off[1], off[1] + ny - 1),
            slice(off[0], off[0] + nx - 1))


def apply_assembled(Ae, x):
    """y = A x where A is assembled from the element matrix Ae over every grid element.

    y at local node a of each element accumulates sum_b Ae[a, b] * x at local node b.
    """
    x = np.asarray(x, dtype=np.float64)
    if min(x.shape) < 2:
        raise ValueError("each axis needs at least 2 nodes")
    y = np.zeros_like(x)
    for a in range(8):
        acc = np.zeros(tuple(s - 1 for s in x.shape))
        for b in range(8):
            if Ae[a, b] != 0.0:
                acc += Ae[a, b] * x[_elem_slice(x.shape, LOCAL[b])]
        y[_elem_slice(x.shape, LOCAL[a])] += acc
    return y


def assembled_diagonal(Ae, shape):
    """Diagonal of the assembled operator: sum of Ae[a, a] over the elements around a node."""
    return apply_assembled(np.diag(np.diag(Ae)), np.ones(shape))


def lumped_mass(shape, h):
    """Lumped nodal volume m_i = sum over elements of int N_i (interior value hx*hy*hz)."""
    ei = element_integrals(h)
    y = np.zeros(shape)
    for a in range(8):
        y[_elem_slice(shape, LOCAL[a])] += ei["lumped"][a]
    return y


def filter_apply(C_padded, w):
    """Generic filter application of Section 2.2.2 (the paper's f(C; w)).

    f(C; w)|_{i,j,k} = sum_{ii,jj,kk=-l..l} w_{ii,jj,kk} C_{i+ii, j+jj, k+kk}, on a tensor padded
    by l halo layers; the output is unpadded.  Here ``w`` is stored [kk, jj, ii] (z, y, x), the
    same slice/row/column layout in which the paper prints its filters.
    """
    w = np.asarray(w, dtype=np.float64)
    l = w.shape[0] // 2
    nz, ny, nx = (s - 2 * l for s in C_padded.shape)
    out = np.zeros((nz, ny, nx))
    for kk in range(-l, l + 1):
        for jj in range(-l, l + 1):
            for ii in range(-l, l + 1):
                c = w[kk + l, jj + l, ii + l]
                if c != 0.0:
                    out += c * C_padded[l + kk:l + kk + nz, l + jj:l + jj + ny, l + ii:l + ii + nx]
    return out


def interior_filter(Ae, h_shape=(5, 5, 5)):
    """The 3x3x3 filter that an assembled operator applies at an interior node.

    Obtained by applying the operator to unit vectors around the centre of a 5^3 grid: the
    column j of A at the centre row gives w_{j - centre}.  Used to compare with printed filters.
    """
    c = tuple(s // 2 for s in h_shape)
    w = np.zeros((3, 3, 3))
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        e = np.zeros(h_shape)
        e[c[0] + dz, c[1] + dy, c[2] + dx] = 1.0
        w[dz + 1, dy + 1, dx + 1] = apply_assembled(Ae, e)[c]
    return w
