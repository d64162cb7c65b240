"""Seeded random complex coefficient vectors (inputs only)."""

import numpy as np


def random_complex(shape, seed=0):
    """Complex128 array with independent standard-normal real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
