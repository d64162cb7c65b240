"""GPU parity for stencil orders 1 and 3 (2x2x2 and 4x4x4 nodes per basis), both
formulations, every product path: FP64 generic 1e-9, FP32 plane-fused and generic
1e-5, against the FP64 oracle's direct grid summation; setup products exact or
to 1e-10 of their scale."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02281_gb300 import build
    build.build()
    return torch


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("form", ["efie", "pmchwt"])
def test_product_parity_other_orders(torch_cuda, order, form):
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE, PMCHWT
    xyz, tri = icosphere(2)
    grid = (16, 16, 16)
    kw = dict(formulation=EFIE) if form == "efie" else dict(formulation=PMCHWT, eps_out=1.0, eps_in=2.5)
    ctx = Context(xyz, tri, grid, order=order, **kw)
    prob = op.setup(xyz, tri, order, grid, radius=3)
    ex = ctx.export_setup()
    assert np.array_equal(ex["anchors"], prob["anc"])
    assert np.array_equal(ex["cols"], prob["cols"])
    assert np.abs(ex["weights"] - prob["lam"]).max() <= 1e-11 * np.abs(prob["lam"]).max()
    for k in ("NA", "NP", "NK"):
        assert np.abs(ex[k] - prob["near"][k]).max() <= 1e-10 * np.abs(prob["near"][k]).max(), k
    f = 1.1 * C0 / (2 * np.pi)
    x = random_complex((3, ctx.nunk), seed=40 + order)
    if form == "efie":
        ref = np.stack([op.matvec_efie(prob, f, v) for v in x])
    else:
        ref = np.stack([op.matvec_pmchwt(prob, f, v, 1.0, 2.5) for v in x])
    y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert _rel(y64, ref) <= 1e-9
    for path, expect in ((0, 0), (1, 1)):
        ctx.set_path(path)
        assert ctx.matvec_path() == expect
        y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
        assert _rel(y32, ref) <= 1e-5, path
    ctx.close()
