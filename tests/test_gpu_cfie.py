"""GPU parity of the AIMx CFIE for closed PEC bodies (Sec. III-B, Eq. CFIEAIMx).

Near K_g values to 1e-10 of their scale (FP64 on both sides), products to the
matvec tolerances (FP64 1e-9, FP32 1e-5) on the generic and cuFFT paths,
plane-wave right-hand sides to 1e-12, and GMRES against the dense oracle
matrix; the CFIE needs fewer iterations than the EFIE on the same sphere.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0


@pytest.fixture(scope="module")
def sphere():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth import icosphere
    from oracle import operator as op, cfie
    from paper_2009_02281_gb300 import build, Context, CFIE
    build.build()
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (12, 12, 12), order=2, formulation=CFIE)
    prob = cfie.setup_cfie(op.setup(xyz, tri, 2, (12, 12, 12), radius=3))
    yield torch, ctx, prob
    ctx.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_setup_parity(sphere):
    torch, ctx, prob = sphere
    ex = ctx.export_setup()
    assert np.array_equal(ex["cols"], prob["cols"])
    for k, ref in (("NA", prob["near"]["NA"]), ("NP", prob["near"]["NP"]), ("NK", prob["near"]["NKG"])):
        assert np.abs(ex[k] - ref).max() <= 1e-10 * np.abs(ref).max(), k
    assert ctx.matvec_path(0) == 1            # generic path


def test_product_parity(sphere):
    torch, ctx, prob = sphere
    from synth import random_complex
    from oracle import cfie
    f = 1.3 * C0 / (2 * np.pi)
    x = random_complex((2, ctx.nunk), seed=23)
    ref = np.stack([cfie.matvec_cfie(prob, f, v) for v in x])
    for path in (1, 2):
        ctx.set_path(path)
        y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
        y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
        assert _rel(y64, ref) <= 1e-9, path
        assert _rel(y32, ref) <= 1e-5, path
    ctx.set_path(0)


def test_rhs_parity(sphere):
    torch, ctx, prob = sphere
    from oracle import cfie
    k = 1.3
    f = k * C0 / (2 * np.pi)
    b = ctx.rhs_planewave(f, [[0.0, 0.6, 0.8]], [[1.0, 0.0, 0.0]]).cpu().numpy()[0]
    ref = cfie.planewave_rhs_cfie(prob["rwg"], k, [0.0, 0.6, 0.8], [1.0, 0.0, 0.0])
    assert _rel(b, ref) <= 1e-12


def test_solve_matches_dense_and_beats_efie(sphere):
    torch, ctx, prob = sphere
    from oracle import cfie
    from paper_2009_02281_gb300 import Context, EFIE, F64
    from synth import icosphere
    k = 1.3
    f = k * C0 / (2 * np.pi)
    b = ctx.rhs_planewave(f, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])
    x, st, rc = ctx.solve(f, b, tol=1e-10, restart=100, max_iter=1000, inner_precision=F64)
    assert rc == 0, st
    Z = cfie.dense_cfie(prob, f)
    xg = x.cpu().numpy()[0]
    bb = b.cpu().numpy()[0]
    assert np.linalg.norm(Z @ xg - bb) <= 1e-8 * np.linalg.norm(bb)
    xyz, tri = icosphere(2)
    e = Context(xyz, tri, (12, 12, 12), order=2, formulation=EFIE)
    be = e.rhs_planewave(f, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])
    _, ste, rce = e.solve(f, be, tol=1e-10, restart=100, max_iter=1000, inner_precision=F64)
    e.close()
    assert rce == 0
    assert st[0]["iterations"] < ste[0]["iterations"]


def test_linear_term_scaled_by_alpha(sphere):
    torch, ctx, prob = sphere
    from synth import random_complex
    from oracle import linterm, operator as op
    f = 1.3 * C0 / (2 * np.pi)
    x = random_complex((1, ctx.nunk), seed=4)
    xt = torch.tensor(x, dtype=torch.complex128, device="cuda")
    off = ctx.matvec(f, xt).cpu().numpy()[0]
    ctx.set_linear_term(True)
    on = ctx.matvec(f, xt).cpu().numpy()[0]
    ctx.set_linear_term(False)
    d_ref = 0.5 * (linterm.matvec_efie_lin(prob, f, x[0]) - op.matvec_efie(prob, f, x[0]))
    assert _rel(on - off, d_ref) <= 1e-7


def test_cfie_errors(sphere):
    torch, ctx, prob = sphere
    from paper_2009_02281_gb300 import AimxError, Context, CFIE, PRECOND_BLOCK
    from synth import icosphere
    f = 1.3 * C0 / (2 * np.pi)
    b = ctx.rhs_planewave(f, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])
    with pytest.raises(AimxError) as e:
        ctx.solve(f, b, precond=PRECOND_BLOCK)
    assert e.value.code == -7
    with pytest.raises(AimxError) as e:
        ctx.set_conventional_aim(True)
    assert e.value.code == -7
    xyz, tri = icosphere(1)
    with pytest.raises(AimxError) as e:
        Context(xyz, tri, (8, 8, 8), formulation=CFIE, cfie_alpha=1.5)
    assert e.value.code == -1


def test_static_roundtrip(sphere, tmp_path):
    torch, ctx, prob = sphere
    from synth import random_complex
    from paper_2009_02281_gb300 import Context
    path = tmp_path / "cfie.aimx"
    ctx.save_static(path)
    c2 = Context.load_static(path)
    f = 1.1 * C0 / (2 * np.pi)
    x = torch.tensor(random_complex((2, ctx.nunk), seed=8), dtype=torch.complex128, device="cuda")
    assert np.array_equal(ctx.matvec(f, x).cpu().numpy(), c2.matvec(f, x).cpu().numpy())
    c2.close()
