"""Seeded plane-wave incidence directions and polarisations (inputs only)."""

import numpy as np


def theta_hat(d):
    """Unit theta vector of direction d (x-hat when d is along +-z)."""
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    rho = np.hypot(d[0], d[1])
    if rho < 1e-12:
        return np.array([1.0, 0.0, 0.0])
    cth, sth = d[2], rho
    cph, sph = d[0] / rho, d[1] / rho
    return np.array([cth * cph, cth * sph, -sth])


def planewave_batch(n_dir, seed=0):
    """``n_dir`` propagation directions drawn uniformly on the unit sphere.

    Directions are normalised standard-normal draws from
    ``numpy.random.default_rng(seed)``; each polarisation is the theta unit
    vector of its direction.  Returns (dirs [n,3], pols [n,3]).
    """
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n_dir, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = np.stack([theta_hat(x) for x in d])
    return d, p
