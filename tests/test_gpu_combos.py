"""GPU parity of option combinations: the surface impedance inside the CFIE (it
enters the EFIE part, weighted by alpha) and inside the conventional-AIM mode
(added to the per-frequency near entries), against the oracle's Gram matrix."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
SIGMA = 5.8e7


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02281_gb300 import build
    build.build()
    return torch


def _gram_apply(prob, x):
    from oracle import sibc
    G = sibc.gram(prob["rwg"], prob["near"]["rows"], prob["cols"])
    y = np.zeros(prob["N"], dtype=np.complex128)
    np.add.at(y, prob["near"]["rows"], G * x[prob["cols"]])
    return y


@pytest.mark.parametrize("mode", ["cfie", "aim"])
def test_surface_impedance_combinations(torch_cuda, mode):
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op, sibc
    from paper_2009_02281_gb300 import Context, CFIE, EFIE
    xyz, tri = icosphere(1)
    grid = (8, 8, 8)
    form = CFIE if mode == "cfie" else EFIE
    a = Context(xyz, tri, grid, order=2, formulation=form)
    b = Context(xyz, tri, grid, order=2, formulation=form, sigma=SIGMA)
    if mode == "aim":
        a.set_conventional_aim(True)
        b.set_conventional_aim(True)
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    f = 1.3 * C0 / (2 * np.pi)
    x = random_complex((2, a.nunk), seed=19)
    xt = torch.tensor(x, dtype=torch.complex128, device="cuda")
    d = (b.matvec(f, xt) - a.matvec(f, xt)).cpu().numpy()
    w = 0.5 if mode == "cfie" else 1.0          # the EFIE weight alpha of the CFIE
    ref = np.stack([w * sibc.surface_impedance(f, SIGMA) * _gram_apply(prob, v) for v in x])
    assert np.linalg.norm(d - ref) <= 1e-9 * np.linalg.norm(ref)
    x32 = torch.tensor(x, dtype=torch.complex64, device="cuda")
    d32 = (b.matvec(f, x32) - a.matvec(f, x32)).cpu().numpy()
    y32 = b.matvec(f, x32).cpu().numpy()
    assert np.linalg.norm(d32 - ref) <= 1e-5 * np.linalg.norm(y32)
    a.close()
    b.close()
