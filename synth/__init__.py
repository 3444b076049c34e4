"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the method itself: only a counter-based random number
generator and the geometric recipes (node coordinates, spheres, columns) that the workloads
are built from.  Both sides of every comparison receive the same host arrays from here.

Generator: splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) used as a counter-based hash.  Stream element ``n`` of seed ``s`` is
``mix(s * 2^32 + n + 1 scaled by the golden gamma)``; uniforms are ``(z >> 11) * 2^-53`` and
standard normals come from the Box-Muller transform of two consecutive uniforms.
"""

from .generators import (  # noqa: F401
    splitmix64,
    uniform01,
    standard_normal,
    node_coords,
    sphere_ramp_field,
    sharp_sphere_field,
    column_field,
)
