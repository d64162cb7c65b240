"""GPU parity of the batched frequency sweep (aimx_sweep_batched).

All frequencies and right-hand sides of a sweep are solved together with device-side GMRES
(Givens rotations and convergence tests on the GPU, one CUDA graph per cycle).  Every solution is
checked against the oracle's dense LU solution of the same AIMx system at its frequency (rel-L2
<= 1e-4, the solved-current tolerance) and against the per-frequency aimx_solve; the reported
true residuals against the requested tolerance and an independent residual with the oracle's
dense operator.  Covered: the EFIE on a grid of the generic path, the two-region form, the
charge-form scalar potential, FP64 inner products, a batch smaller than the sweep (pending
systems admitted as slots free up, the batch shrinking to fewer slots), no preconditioner, and
the refused combinations.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
ETA0 = 4e-7 * np.pi * C0


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02281_gb300 import build
    build.build()
    return torch


def _rhs_all(ctx, freqs, dirs, pols, torch):
    return torch.stack([ctx.rhs_planewave(f, dirs, pols) for f in freqs])


def _oracle_rhs(prob, f, d, p, two_region=False):
    from oracle import excitation
    k = 2 * np.pi * f / C0
    if two_region:
        VE, VH = excitation.planewave_rhs(prob["rwg"], k, d, p, eta=ETA0)
        return np.r_[VE, ETA0 * VH]
    return excitation.planewave_rhs(prob["rwg"], k, d, p)[0]


@pytest.fixture(scope="module")
def efie12(torch_cuda):
    """Level-2 icosphere, 12^3 grid (padded 24^3 = 3 * 8 per axis: the generic path)."""
    from synth import icosphere
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE, F32
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (12, 12, 12), order=2, formulation=EFIE)
    assert ctx.matvec_path(F32) == 1
    prob = op.setup(xyz, tri, 2, (12, 12, 12), radius=3)
    yield ctx, prob
    ctx.close()


@pytest.mark.parametrize("inner,max_batch", [("f32", 0), ("f64", 0), ("f32", 4)])
def test_efie_sweep_matches_lu_and_solve(efie12, torch_cuda, inner, max_batch):
    torch = torch_cuda
    from synth import planewave_batch
    from oracle import operator as op, solve as osolve
    from paper_2009_02281_gb300 import F32, F64
    ctx, prob = efie12
    freqs = np.array([0.5, 0.8, 1.1, 1.4, 1.7, 2.0]) * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(2, seed=11)
    B = _rhs_all(ctx, freqs, dirs, pols, torch)
    tol = 1e-9
    prec = F32 if inner == "f32" else F64
    X, stats, rc, cnt = ctx.sweep_batched(freqs, B, tol=tol, restart=40, inner_precision=prec,
                                          max_batch=max_batch)
    assert rc == 0, stats
    cycles, graphs, products = cnt
    assert cycles >= 1 and 1 <= graphs <= cycles and products > cycles
    if max_batch:
        assert graphs >= 1
    Xh = X.cpu().numpy()
    for i, f in enumerate(freqs):
        Z = op.dense_efie(prob, f)
        for w in range(2):
            assert stats[i][w]["rel_residual"] <= tol
            bn = _oracle_rhs(prob, f, dirs[w], pols[w])
            assert _rel(Xh[i, w], osolve.lu_solve(Z, bn)) <= 1e-4
            assert np.linalg.norm(Z @ Xh[i, w] - bn) / np.linalg.norm(bn) <= 10 * tol
    # the per-frequency solver reaches the same solutions
    for i in (0, len(freqs) - 1):
        x, _, _ = ctx.solve(freqs[i], B[i], tol=tol, inner_precision=prec)
        assert _rel(Xh[i], x.cpu().numpy()) <= 1e-6


def test_pmchwt_sweep_matches_lu(torch_cuda):
    torch = torch_cuda
    from synth import icosphere, planewave_batch
    from oracle import operator as op, solve as osolve
    from paper_2009_02281_gb300 import Context, PMCHWT
    xyz, tri = icosphere(2)
    grid = (12, 12, 12)
    ctx = Context(xyz, tri, grid, order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    freqs = np.array([0.7, 1.3]) * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(2, seed=12)
    B = _rhs_all(ctx, freqs, dirs, pols, torch)
    tol = 1e-9
    X, stats, rc, _ = ctx.sweep_batched(freqs, B, tol=tol, restart=60)
    Xh = X.cpu().numpy()
    ctx.close()
    assert rc == 0, stats
    for i, f in enumerate(freqs):
        Z = op.dense_pmchwt(prob, f, 1.0, 4.0)
        for w in range(2):
            bn = _oracle_rhs(prob, f, dirs[w], pols[w], two_region=True)
            assert _rel(Xh[i, w], osolve.lu_solve(Z, bn)) <= 1e-4


def test_charge_form_sweep_matches_lu(efie12, torch_cuda):
    torch = torch_cuda
    from synth import planewave_batch
    from oracle import chargepot as cp, solve as osolve
    ctx, prob = efie12
    ctx.set_charge_form(True)
    try:
        ch = cp.setup_charge(prob)
        freqs = np.array([0.4, 0.9, 1.6]) * C0 / (2 * np.pi)
        dirs, pols = planewave_batch(1, seed=13)
        B = _rhs_all(ctx, freqs, dirs, pols, torch)
        tol = 1e-9
        X, stats, rc, _ = ctx.sweep_batched(freqs, B, tol=tol, restart=60, max_iter=3000)
        assert rc == 0, stats
        Xh = X.cpu().numpy()
        for i, f in enumerate(freqs):
            Z = cp.dense_efie_charge(prob, ch, f)
            bn = _oracle_rhs(prob, f, dirs[0], pols[0])
            assert _rel(Xh[i, 0], osolve.lu_solve(Z, bn)) <= 1e-4
    finally:
        ctx.set_charge_form(False)


def test_no_preconditioner_and_errors(efie12, torch_cuda):
    torch = torch_cuda
    from synth import planewave_batch
    from paper_2009_02281_gb300 import AimxError, PRECOND_NONE, PRECOND_BLOCK
    ctx, prob = efie12
    freqs = np.array([0.9, 1.2]) * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(1, seed=14)
    B = _rhs_all(ctx, freqs, dirs, pols, torch)
    X, stats, rc, _ = ctx.sweep_batched(freqs, B, tol=1e-8, restart=80, max_iter=3000, precond=PRECOND_NONE)
    assert rc == 0
    for i, f in enumerate(freqs):
        x, _, _ = ctx.solve(f, B[i], tol=1e-8)
        assert _rel(X[i].cpu().numpy(), x.cpu().numpy()) <= 1e-5
    with pytest.raises(AimxError) as e:
        ctx.sweep_batched(freqs, B, precond=PRECOND_BLOCK)
    assert e.value.code == -7
    # a cap that is too small is a positive warning with per-system status
    X, stats, rc, _ = ctx.sweep_batched(freqs, B, tol=1e-13, restart=3, max_iter=3)
    assert rc == 1 and all(s["status"] == 1 for row in stats for s in row)


def test_warm_start_fewer_iterations(efie12, torch_cuda):
    """Interleaved admission with warm starts from converged neighbours: the same solutions
    (dense LU), fewer iterations in total than cold starts."""
    torch = torch_cuda
    from oracle import operator as op, solve as osolve
    ctx, prob = efie12
    freqs = np.linspace(0.8, 1.6, 12) * C0 / (2 * np.pi)
    d, p = [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]]
    B = _rhs_all(ctx, freqs, d, p, torch)
    tol = 1e-9
    Xc, sc, rc, _ = ctx.sweep_batched(freqs, B, tol=tol, restart=40, max_batch=6)
    Xw, sw, rw, _ = ctx.sweep_batched(freqs, B, tol=tol, restart=40, max_batch=6, warm_start=True)
    assert rc == 0 and rw == 0
    cold = sum(s["iterations"] for row in sc for s in row)
    warm = sum(s["iterations"] for row in sw for s in row)
    assert warm < cold, (warm, cold)
    Xh = Xw.cpu().numpy()
    for i in (0, 5, 11):
        Z = op.dense_efie(prob, freqs[i])
        ref = osolve.lu_solve(Z, _oracle_rhs(prob, freqs[i], d[0], p[0]))
        assert _rel(Xh[i, 0], ref) <= 1e-4
