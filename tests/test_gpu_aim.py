"""GPU parity of the conventional-AIM comparison mode (Sec. II-B).

Per-frequency near entries j w mu (N^A(k) - k^-2 N^Phi(k)) against the oracle
to 1e-10 of their scale (FP64 on both sides, the same quadrature); products
with the mode on to the matvec tolerances (FP64 1e-9, FP32 1e-5) on both FP32
paths and across a frequency change; GMRES against the dense oracle matrix.
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
    from oracle import operator as op
    from paper_2009_02281_gb300 import build, Context, EFIE
    build.build()
    xyz, tri = icosphere(1)
    ctx = Context(xyz, tri, (8, 8, 8), order=2, formulation=EFIE)
    prob = op.setup(xyz, tri, 2, (8, 8, 8), radius=3)
    yield torch, ctx, prob
    ctx.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _z_oracle(prob, f):
    from oracle import aim
    w = 2 * np.pi * f
    k = w / C0
    mu = 4e-7 * np.pi
    NA, NP = aim.near_aim(prob, k)
    return 1j * w * mu * (NA - NP / k ** 2), (NA, NP)


def test_state_errors(sphere):
    torch, ctx, _ = sphere
    from paper_2009_02281_gb300 import AimxError, Context, PMCHWT
    from synth import icosphere
    with pytest.raises(AimxError) as e:
        ctx.export_aim_near(1e8)
    assert e.value.code == -7
    xyz, tri = icosphere(1)
    c = Context(xyz, tri, (8, 8, 8), formulation=PMCHWT, eps_in=2.0)
    with pytest.raises(AimxError) as e:
        c.set_conventional_aim(True)
    assert e.value.code == -7
    c.close()


@pytest.mark.parametrize("ka", [0.5, 1.7])
def test_near_entries_match_oracle(sphere, ka):
    torch, ctx, prob = sphere
    f = ka * C0 / (2 * np.pi)
    ctx.set_conventional_aim(True)
    z = ctx.export_aim_near(f)
    ref, _ = _z_oracle(prob, f)
    assert np.abs(z - ref).max() <= 1e-10 * np.abs(ref).max()


def test_products_match_oracle_across_frequencies(sphere):
    torch, ctx, prob = sphere
    from synth import random_complex
    from oracle import aim
    ctx.set_conventional_aim(True)
    x = random_complex((2, ctx.nunk), seed=41)
    for ka in (0.9, 1.4, 0.9):
        f = ka * C0 / (2 * np.pi)
        _, near = _z_oracle(prob, f)
        ref = np.stack([aim.matvec_efie_aim(prob, f, v, near=near) for v in x])
        y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
        assert _rel(y64, ref) <= 1e-9, ka
        for path in (0, 1):
            ctx.set_path(path)
            y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
            assert _rel(y32, ref) <= 1e-5, (ka, path)
        ctx.set_path(0)


def test_toggle_returns_to_aimx(sphere):
    torch, ctx, prob = sphere
    from synth import random_complex
    from oracle import operator as op
    f = 1.2 * C0 / (2 * np.pi)
    x = random_complex((1, ctx.nunk), seed=3)
    xt = torch.tensor(x, dtype=torch.complex128, device="cuda")
    ctx.set_conventional_aim(True)
    on = ctx.matvec(f, xt).cpu().numpy()[0]
    ctx.set_conventional_aim(False)
    off = ctx.matvec(f, xt).cpu().numpy()[0]
    assert _rel(off, op.matvec_efie(prob, f, x[0])) <= 1e-9
    assert _rel(on, off) > 1e-5


def test_solve_matches_dense(sphere):
    torch, ctx, prob = sphere
    from synth import random_complex
    from oracle import aim
    from paper_2009_02281_gb300 import F64
    f = 1.1 * C0 / (2 * np.pi)
    ctx.set_conventional_aim(True)
    _, near = _z_oracle(prob, f)
    Z = aim.dense_efie_aim(prob, f, near=near)
    b = random_complex((1, ctx.nunk), seed=17)
    # restart above the 120 unknowns: full GMRES
    x, stats, rc = ctx.solve(f, torch.tensor(b, dtype=torch.complex128, device="cuda"), tol=1e-10,
                             restart=150, max_iter=1000, inner_precision=F64)
    ctx.set_conventional_aim(False)
    assert rc == 0, stats
    xg = x.cpu().numpy()[0]
    assert np.linalg.norm(Z @ xg - b[0]) <= 1e-8 * np.linalg.norm(b[0])
