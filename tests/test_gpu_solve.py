"""GPU parity of the right-hand sides, far field, iterative solve and sweep.

Solved currents are compared with the oracle's dense LU solution of the same
AIMx system (rel-L2 <= 1e-4, the solved-current tolerance); the true relative
residual reported by the solver is checked against the requested tolerance;
the 1920-unknown PEC sphere at ka = pi is compared with the Mie series.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
ETA0 = 4e-7 * np.pi * C0


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02281_gb300 import build
    build.build()
    return torch


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _oracle_rhs(prob, f, dirs, pols, two_region=False):
    """Plane-wave right-hand sides computed by the oracle (never taken from the GPU path)."""
    from oracle import excitation
    k = 2 * np.pi * f / C0
    out = []
    for d, p in zip(np.atleast_2d(dirs), np.atleast_2d(pols)):
        if two_region:
            VE, VH = excitation.planewave_rhs(prob["rwg"], k, d, p, eta=ETA0)
            out.append(np.r_[VE, ETA0 * VH])
        else:
            VE, _ = excitation.planewave_rhs(prob["rwg"], k, d, p)
            out.append(VE)
    return np.array(out)


@pytest.fixture(scope="module")
def efie_l2(torch_cuda):
    from synth import icosphere
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (16, 16, 16), order=2, formulation=EFIE)
    prob = op.setup(xyz, tri, 2, (16, 16, 16), radius=3)
    yield ctx, prob
    ctx.close()


@pytest.fixture(scope="module")
def pmchwt_l2(torch_cuda):
    from synth import icosphere
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, PMCHWT
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (16, 16, 16), order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    prob = op.setup(xyz, tri, 2, (16, 16, 16), radius=3)
    yield ctx, prob
    ctx.close()


def test_rhs_parity(efie_l2, pmchwt_l2):
    from synth import planewave_batch
    from oracle import excitation
    dirs, pols = planewave_batch(3, seed=4)
    k = 1.3
    f = k * C0 / (2 * np.pi)
    ctx, prob = efie_l2
    b = ctx.rhs_planewave(f, dirs, pols).cpu().numpy()
    for w in range(3):
        ref, _ = excitation.planewave_rhs(prob["rwg"], k, dirs[w], pols[w])
        assert _relerr(b[w], ref) <= 1e-12
    ctx, prob = pmchwt_l2
    b = ctx.rhs_planewave(f, dirs, pols).cpu().numpy()
    N = ctx.N
    for w in range(3):
        VE, VH = excitation.planewave_rhs(prob["rwg"], k, dirs[w], pols[w], eta=ETA0)
        assert _relerr(b[w], np.r_[VE, ETA0 * VH]) <= 1e-12


def test_farfield_parity(pmchwt_l2, torch_cuda):
    torch = torch_cuda
    from synth import random_complex
    from oracle import farfield
    from oracle.constants import MU0
    ctx, prob = pmchwt_l2
    N = ctx.N
    x = random_complex((2, ctx.nunk), seed=6)
    k = 0.9
    f = k * C0 / (2 * np.pi)
    th = np.linspace(0.1, 3.0, 5)
    dirs = np.stack([np.sin(th), 0.3 * np.sin(th), np.cos(th)], 1)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    E = ctx.farfield(f, torch.tensor(x, device="cuda"), dirs)
    for b in range(2):
        ref = farfield.far_field(prob["rwg"], x[b, :N], k, 2 * np.pi * f, MU0, dirs, M=ETA0 * x[b, N:])
        assert _relerr(E[b], ref) <= 1e-12


@pytest.mark.parametrize("inner", ["f32", "f64"])
def test_efie_solve_matches_lu(efie_l2, torch_cuda, inner):
    torch = torch_cuda
    from synth import planewave_batch
    from oracle import operator as op, solve as osolve
    from paper_2009_02281_gb300 import F32, F64
    ctx, prob = efie_l2
    k = 1.7
    f = k * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(2, seed=1)
    b = ctx.rhs_planewave(f, dirs, pols)
    tol = 1e-9
    x, stats, rc = ctx.solve(f, b, tol=tol, restart=60, inner_precision=F32 if inner == "f32" else F64)
    assert rc == 0, stats
    Z = op.dense_efie(prob, f)
    bn = _oracle_rhs(prob, f, dirs, pols)
    for w in range(2):
        assert stats[w]["rel_residual"] <= tol
        ref = osolve.lu_solve(Z, bn[w])
        assert _relerr(x.cpu().numpy()[w], ref) <= 1e-4
        # independent residual check with the oracle's dense operator
        assert np.linalg.norm(Z @ x.cpu().numpy()[w] - bn[w]) / np.linalg.norm(bn[w]) <= 10 * tol


def test_pmchwt_solve_matches_lu(pmchwt_l2, torch_cuda):
    from synth import planewave_batch
    from oracle import operator as op, solve as osolve
    ctx, prob = pmchwt_l2
    k = 0.8
    f = k * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(3, seed=2)
    b = ctx.rhs_planewave(f, dirs, pols)
    x, stats, rc = ctx.solve(f, b, tol=1e-9, restart=60)
    assert rc == 0, stats
    Z = op.dense_pmchwt(prob, f, 1.0, 4.0)
    bn = _oracle_rhs(prob, f, dirs, pols, two_region=True)
    for w in range(3):
        ref = osolve.lu_solve(Z, bn[w])
        assert _relerr(x.cpu().numpy()[w], ref) <= 1e-4


def test_batched_equals_single(efie_l2, torch_cuda):
    from synth import planewave_batch
    ctx, _ = efie_l2
    f = 1.1 * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(3, seed=9)
    b = ctx.rhs_planewave(f, dirs, pols)
    xb, sb, rc = ctx.solve(f, b, tol=1e-10)
    assert rc == 0
    for w in range(3):
        xs, ss, rc1 = ctx.solve(f, b[w:w + 1], tol=1e-10)
        assert rc1 == 0
        assert _relerr(xs.cpu().numpy()[0], xb.cpu().numpy()[w]) <= 1e-7


def test_sweep_matches_individual_solves(efie_l2, torch_cuda):
    from synth import planewave_batch
    ctx, _ = efie_l2
    freqs = np.array([0.6, 1.0, 1.5]) * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(2, seed=3)
    X, stats, rc = ctx.sweep(freqs, dirs, pols, tol=1e-9)
    assert rc == 0
    assert all(s["rel_residual"] <= 1e-9 for s in stats)
    for i, f in enumerate(freqs):
        b = ctx.rhs_planewave(f, dirs, pols)
        x, _, _ = ctx.solve(f, b, tol=1e-9)
        assert _relerr(X[i].cpu().numpy(), x.cpu().numpy()) <= 1e-6


def test_nonconvergence_reported(efie_l2):
    """An iteration cap that is too small returns the positive warning, not an error."""
    from synth import planewave_batch
    ctx, _ = efie_l2
    f = 1.2 * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(1, seed=5)
    b = ctx.rhs_planewave(f, dirs, pols)
    x, stats, rc = ctx.solve(f, b, tol=1e-12, restart=5, max_iter=5, max_refine=1)
    assert rc == 1
    assert stats[0]["status"] == 1 and stats[0]["iterations"] <= 5


def test_pec_sphere_1920_mie_and_lu(torch_cuda):
    """The plain-method workload: PEC sphere, 1920 RWG, 24^3 grid, ka = pi, x-polarised wave along +z."""
    torch = torch_cuda
    from synth import workloads
    from oracle import operator as op, solve as osolve, mie, farfield
    from oracle.constants import MU0
    from paper_2009_02281_gb300 import Context, EFIE
    wl = workloads.pec_sphere_1920()
    ctx = Context(wl["xyz"], wl["tri"], wl["grid_n"], order=2, formulation=EFIE)
    f = wl["freq"]
    k = 2 * np.pi * f / C0
    b = ctx.rhs_planewave(f, [[0, 0, 1.0]], [[1.0, 0, 0]])
    x, stats, rc = ctx.solve(f, b, tol=1e-8, restart=100)
    assert rc == 0 and stats[0]["rel_residual"] <= 1e-8
    prob = op.setup(wl["xyz"], wl["tri"], 2, wl["grid_n"], radius=3)
    Z = op.dense_efie(prob, f)
    ref = osolve.lu_solve(Z, _oracle_rhs(prob, f, [[0, 0, 1.0]], [[1.0, 0, 0]])[0])
    assert _relerr(x.cpu().numpy()[0], ref) <= 1e-4
    th = np.linspace(0.3, np.pi - 0.3, 7)
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    E = ctx.farfield(f, x, dirs)[0]
    Eo = farfield.far_field(prob["rwg"], ref, k, 2 * np.pi * f, MU0, dirs)
    assert _relerr(E, Eo) <= 1e-4
    s = 4 * np.pi * np.sum(np.abs(E) ** 2, axis=1)
    ref_mie = mie.bistatic_rcs(k, 1.0, th, 0.0)
    assert np.max(np.abs(s - ref_mie)) / ref_mie.max() < 0.08
    ctx.close()


def _block_partition(anc, nx, ny):
    """Bases grouped by 2x2x2 anchor cells in the library's internal order, at most 32 per block."""
    N = len(anc)
    key = (anc[:, 2] * ny + anc[:, 1]) * nx + anc[:, 0]
    internal = np.argsort(key, kind="stable")
    cx, cy = (nx + 1) // 2, (ny + 1) // 2
    ck = ((anc[internal, 2] >> 1) * cy + (anc[internal, 1] >> 1)) * cx + (anc[internal, 0] >> 1)
    order = internal[np.argsort(ck, kind="stable")]
    cks = np.sort(ck, kind="stable")
    blocks = []
    start = 0
    for i in range(1, N + 1):
        if i == N or cks[i] != cks[start]:
            grp = order[start:i]
            blocks += [grp[j:j + 32] for j in range(0, len(grp), 32)]
            start = i
    return blocks


@pytest.mark.parametrize("form", ["efie", "pmchwt"])
def test_block_preconditioner_matches_dense_blocks(efie_l2, pmchwt_l2, torch_cuda, form):
    """M v equals the inverse of the dense AIMx matrix's diagonal blocks applied to v (FP32 inverse)."""
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import PRECOND_BLOCK
    ctx, prob = efie_l2 if form == "efie" else pmchwt_l2
    f = 1.3 * C0 / (2 * np.pi)
    Z = op.dense_efie(prob, f) if form == "efie" else op.dense_pmchwt(prob, f, 1.0, 4.0)
    v = random_complex((2, ctx.nunk), seed=12)
    z = ctx.precond_apply(f, torch.tensor(v, device="cuda"), PRECOND_BLOCK).cpu().numpy()
    N = ctx.N
    ref = np.zeros_like(v)
    for blk in _block_partition(prob["anc"], 16, 16):
        idx = blk if form == "efie" else np.r_[blk, N + blk]
        ref[:, idx] = np.linalg.solve(Z[np.ix_(idx, idx)], v[:, idx].T).T
    assert _relerr(z, ref) <= 1e-4


def test_block_preconditioned_solve_matches_lu(pmchwt_l2, torch_cuda):
    """Solves with the block preconditioner reach the same currents (its iteration count is not asserted:
    on these spheres the oracle's exact-arithmetic GMRES also needs more iterations with 2x2x2-cell blocks
    than with the paper's diagonal)."""
    from synth import planewave_batch
    from oracle import operator as op, solve as osolve
    from paper_2009_02281_gb300 import PRECOND_BLOCK
    ctx, prob = pmchwt_l2
    f = 1.0 * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(2, seed=8)
    b = ctx.rhs_planewave(f, dirs, pols)
    xb, sbk, rcb = ctx.solve(f, b, tol=1e-8, precond=PRECOND_BLOCK)
    assert rcb == 0
    Z = op.dense_pmchwt(prob, f, 1.0, 4.0)
    bn = _oracle_rhs(prob, f, dirs, pols, two_region=True)
    for w in range(2):
        assert _relerr(xb.cpu().numpy()[w], osolve.lu_solve(Z, bn[w])) <= 1e-4
