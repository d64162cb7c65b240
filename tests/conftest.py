import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU oracle checks")


@pytest.fixture(scope="session")
def small_sphere():
    """Level-1 icosphere (80 triangles, 120 RWG), 8^3 grid, order 2, radius 3."""
    from synth import icosphere
    from oracle import operator as op
    xyz, tri = icosphere(1)
    return op.setup(xyz, tri, 2, [8, 8, 8], radius=3)


@pytest.fixture(scope="session")
def sphere_l2():
    """Level-2 icosphere (320 triangles, 480 RWG), 12^3 grid, order 2, radius 3."""
    from synth import icosphere
    from oracle import operator as op
    xyz, tri = icosphere(2)
    return op.setup(xyz, tri, 2, [12, 12, 12], radius=3)
