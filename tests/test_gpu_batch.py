"""GPU checks of batches of uneven meshes (aimx_batch_*).

The batch runs each member's own FP32 product kernels (on internal streams,
captured in one CUDA graph), so every member's output must equal, bit for bit,
what aimx_matvec gives for that member alone; the first member is also checked
against the oracle's direct-summation product (FP32 tolerance 1e-5).  Graph
replay after the inputs change in place, recapture after a size change, and a
member forced onto the generic path are covered.
"""

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


def _members():
    from synth import icosphere, box, torus
    from paper_2009_02281_gb300 import Context, EFIE, PMCHWT
    ms = []
    xyz, tri = icosphere(2)
    ms.append((Context(xyz, tri, (16, 16, 16), formulation=EFIE), 2.0e8, 3))
    xyz, tri = box([0, 0, 0], [2.0, 1.0, 0.5], [8, 4, 2])
    ms.append((Context(xyz, tri, (32, 16, 8), formulation=PMCHWT, eps_in=3.0), 1.5e8, 1))
    xyz, tri = torus(1.0, 0.35, 24, 10)
    ms.append((Context(xyz, tri, (32, 32, 16), formulation=EFIE), 2.5e8, 2))
    xyz, tri = icosphere(1)
    ms.append((Context(xyz, tri, (8, 8, 8), formulation=PMCHWT, eps_in=2.5), 1.0e8, 4))
    xyz, tri = icosphere(2, radius=0.7)
    c = Context(xyz, tri, (16, 16, 16), formulation=EFIE)
    c.set_path(1)                          # generic FFT path inside the graph
    ms.append((c, 3.0e8, 2))
    return ms


def test_batch_equals_individual_products(torch_cuda):
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    from synth import icosphere
    from paper_2009_02281_gb300 import Batch
    ms = _members()
    ctxs = [m[0] for m in ms]
    freqs = [m[1] for m in ms]
    xs = [torch.tensor(random_complex((m[2], m[0].nunk), seed=10 + i), dtype=torch.complex64, device="cuda")
          for i, m in enumerate(ms)]
    ys = [torch.empty_like(x) for x in xs]
    batch = Batch(ctxs, nstreams=3)
    batch.matvec(freqs, xs, ys)
    torch.cuda.synchronize()
    assert batch.graph_nodes > 0
    for c, f, x, y in zip(ctxs, freqs, xs, ys):
        ref = c.matvec(f, x).cpu().numpy()
        assert np.array_equal(y.cpu().numpy(), ref)
    # member 0 against the oracle
    xyz, tri = icosphere(2)
    prob = op.setup(xyz, tri, 2, (16, 16, 16), radius=3)
    x0 = xs[0].cpu().numpy().astype(np.complex128)
    ref0 = np.stack([op.matvec_efie(prob, freqs[0], v) for v in x0])
    y0 = ys[0].cpu().numpy()
    assert np.linalg.norm(y0 - ref0) <= 1e-5 * np.linalg.norm(ref0)
    # replay: new values in the same buffers
    for i, x in enumerate(xs):
        x.copy_(torch.tensor(random_complex(tuple(x.shape), seed=50 + i), dtype=torch.complex64, device="cuda"))
    nodes = batch.graph_nodes
    batch.matvec(freqs, xs, ys)
    torch.cuda.synchronize()
    assert batch.graph_nodes == nodes
    for c, f, x, y in zip(ctxs, freqs, xs, ys):
        assert np.array_equal(y.cpu().numpy(), c.matvec(f, x).cpu().numpy())
    # a different right-hand-side count recaptures
    xs[1] = torch.tensor(random_complex((3, ctxs[1].nunk), seed=99), dtype=torch.complex64, device="cuda")
    ys[1] = torch.empty_like(xs[1])
    batch.matvec(freqs, xs, ys)
    torch.cuda.synchronize()
    assert np.array_equal(ys[1].cpu().numpy(), ctxs[1].matvec(freqs[1], xs[1]).cpu().numpy())
    batch.close()
    for c in ctxs:
        c.close()


def test_batch_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2009_02281_gb300 import Batch, AimxError
    ms = _members()[:2]
    batch = Batch([m[0] for m in ms])
    xs = [torch.zeros((1, m[0].nunk), dtype=torch.complex64, device="cuda") for m in ms]
    with pytest.raises(AimxError) as ei:
        batch.matvec([1e8, -1.0], xs, [torch.empty_like(x) for x in xs])
    assert ei.value.code == -1
    batch.close()
    for m in ms:
        m[0].close()


def test_batch_solve_matches_member_solves(torch_cuda):
    """aimx_batch_solve (members' GMRES overlapped on internal streams and host threads) gives
    each member what its own aimx_solve gives, with the reported true residuals within tol."""
    torch = torch_cuda
    from synth import planewave_batch
    from paper_2009_02281_gb300 import Batch
    ms = _members()
    ctxs = [m[0] for m in ms]
    freqs = [m[1] for m in ms]
    bs = []
    for i, (c, f, nr) in enumerate(ms):
        dirs, pols = planewave_batch(nr, seed=40 + i)
        bs.append(c.rhs_planewave(f, dirs, pols))
    tol = 1e-6
    batch = Batch(ctxs, nstreams=3)
    xs, stats, rc = batch.solve(freqs, bs, tol=tol, restart=60, max_iter=3000)
    worst = 0
    for i, (c, f, nr) in enumerate(ms):
        x, st, rc1 = c.solve(f, bs[i], tol=tol, restart=60, max_iter=3000)
        worst = max(worst, rc1)
        # the same solver on the same data: the same iterations, residuals and solutions
        assert [s["iterations"] for s in stats[i]] == [s["iterations"] for s in st], i
        for s, s1 in zip(stats[i], st):
            assert s["status"] == s1["status"]
            assert s["status"] != 0 or s["rel_residual"] <= tol
        a, b = xs[i].cpu().numpy(), x.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b), i
    assert rc == worst
    batch.close()
    for c in ctxs:
        c.close()
