"""Seeded synthetic inputs shared by the FP64 oracle and the GPU library tests.

This package holds only input generation: triangle meshes (icosphere, box,
torus), plane-wave incidence directions and polarisations, and random
coefficient vectors.  It contains none of the method's arithmetic (no RWG
construction, no grid, no Green's function, no quadrature), so that the oracle
and the CUDA path can both consume the same inputs without sharing any code
that computes a result.
"""

from .meshes import icosphere, box, torus, merge_meshes  # noqa: F401
from .excitation import planewave_batch, theta_hat  # noqa: F401
from .vectors import random_complex  # noqa: F401
