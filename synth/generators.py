"""Counter-based random streams and geometric field recipes (no arithmetic of the method)."""

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counters):
    """splitmix64 output for state ``seed * 2^32 + counter`` (vectorised over ``counters``)."""
    c = np.asarray(counters, dtype=np.uint64)
    base = np.uint64((int(seed) << 32) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = (base + c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z & _MASK


def uniform01(seed, n, offset=0):
    """``n`` uniforms in [0, 1) with 53 random bits: ``(z >> 11) * 2^-53``."""
    z = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def standard_normal(seed, n):
    """``n`` N(0,1) samples; sample i uses counters 2i (radius) and 2i+1 (angle)."""
    z = splitmix64(seed, np.arange(2 * n, dtype=np.uint64))
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u1 = u[0::2] + 2.0 ** -53          # in (0, 1]: log is finite
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def node_coords(n, h):
    """Node coordinates of a vertex grid with ``n=(nx,ny,nz)`` nodes and spacing ``h``.

    Returns three arrays of shape (nz, ny, nx) (x fastest), node i of an axis at i*h.
    """
    nx, ny, nz = n
    z = np.arange(nz)[:, None, None] * h[2]
    y = np.arange(ny)[None, :, None] * h[1]
    x = np.arange(nx)[None, None, :] * h[0]
    shape = (nz, ny, nx)
    return (np.broadcast_to(x, shape).copy(), np.broadcast_to(y, shape).copy(),
            np.broadcast_to(z, shape).copy())


def sphere_ramp_field(n, h, centre, radius, width):
    """Indicator that is 0 inside a sphere and 1 outside, with a linear ramp of ``width``.

    value = clamp(1/2 + (r - R) / width, 0, 1), r the distance of the node to ``centre``.
    """
    x, y, z = node_coords(n, h)
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    return np.clip(0.5 + (r - radius) / width, 0.0, 1.0)


def sharp_sphere_field(n, h, centre, radius):
    """Indicator that is 0 at nodes strictly inside the sphere and 1 elsewhere."""
    x, y, z = node_coords(n, h)
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return np.where(r2 < radius * radius, 0.0, 1.0)


def column_field(n, h, xmax, zmax):
    """Indicator that is 1 at nodes with x <= xmax and z <= zmax (inclusive), 0 elsewhere."""
    x, _, z = node_coords(n, h)
    eps = 1e-12
    return np.where((x <= xmax + eps) & (z <= zmax + eps), 1.0, 0.0)
