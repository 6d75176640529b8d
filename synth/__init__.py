"""Seeded synthetic inputs for the carousel phase-retrieval path.

This module builds the measurements a CXDI experiment would record: an
ellipsoid-union density, its projections about the z axis, and the
Poisson-noisy far-field intensities of those projections (the forward model
of Eq. 1-3).  It holds none of the reconstruction arithmetic; both the FP64
oracle and the GPU library consume what it produces, and neither depends on
the other.

Shapes and conventions
  * volume  [z][y][x], centre at index N/2 on every axis;
  * projection image [z][u] (rows = rotation axis z, columns = u), centre at
    index N/2; angles theta_n = n * pi / Np, n = 0..Np-1;
  * intensities are centred (q = 0 at pixel (N/2, N/2)), float32.
"""
from .phantom import (  # noqa: F401
    ellipsoid_phantom,
    pad_volume,
    project,
    intensities,
    padded_box_support,
    angles,
    make_case,
    CASES,
)
