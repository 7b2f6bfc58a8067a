"""Seeded synthetic inputs shared by the CPU oracle and the GPU library tests.

This module only draws random numbers and shapes them into lattice fields; it holds none of
the Dirac-operator, solver, projection, loop or correlator arithmetic.  Everything here is
deterministic in (seed, shape):

* ``philox4x32_10``       counter-based generator of Salmon, Moraes, Dror and Shaw,
                          "Parallel random numbers: as easy as 1, 2, 3" (SC 2011).
* ``gaussians``           Box-Muller normals from Philox output, keyed by (seed, purpose, index).
* ``gauge_field``         SU(3) links U = exp(i eps H), H = sum_a h_a lambda_a / 2, h_a ~ N(0,1).
* ``random_gauge_transform``  a field of SU(3) matrices G(x) (same recipe).
* ``colour_vectors``      complex Gaussian colour vectors, orthonormalised per timeslice.
* ``random_spinors``      complex Gaussian spinor fields.

Array conventions (shared by both sides, fixed here):

* lattice extents ``dims = (Lx, Ly, Lz, Lt)``; a site field is a numpy array of shape
  ``(Lt, Lz, Ly, Lx, ...)`` so the flat site index is ``s = x + Lx*(y + Ly*(z + Lz*t))``;
* links ``U[t, z, y, x, mu, a, b]`` with ``mu = 0..3 = x, y, z, t`` (complex128);
* spinors ``psi[..., t, z, y, x, spin, colour]`` (complex128);
* colour vectors ``V[t, i, z, y, x, colour]`` (complex128).
"""
from .philox import philox4x32_10, gaussians, uniforms
from .fields import (
    gauge_field,
    unit_gauge_field,
    random_gauge_transform,
    colour_vectors,
    random_spinors,
    gell_mann,
    PURPOSE_GAUGE,
    PURPOSE_COLOUR,
    PURPOSE_SPINOR,
    PURPOSE_GAUGE_TRANSFORM,
)

__all__ = [
    "philox4x32_10",
    "gaussians",
    "uniforms",
    "gauge_field",
    "unit_gauge_field",
    "random_gauge_transform",
    "colour_vectors",
    "random_spinors",
    "gell_mann",
    "PURPOSE_GAUGE",
    "PURPOSE_COLOUR",
    "PURPOSE_SPINOR",
    "PURPOSE_GAUGE_TRANSFORM",
]
