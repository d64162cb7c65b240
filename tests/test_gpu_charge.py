"""GPU parity of the charge-form scalar potential (L^Phi = D^T Pt D with Pt in AIMx form),
for the EFIE and for both regions of the PMCHWT.

Setup against the oracle (``oracle/chargepot.py``, pinned by its own CPU tests): triangle
anchors and the triangle near pattern bit-exact, pulse weights and the static near values
N_Pt = Pt_s,NR - Pt_s,P to 1e-12 / 1e-10 of their scale (FP64 on both sides, the same
quadrature).  Products against ``matvec_efie_charge`` at the matvec tolerances (FP64 1e-9,
FP32 1e-5) on the generic and plane-fused paths, several RHS counts (a ragged 32-RHS chunk),
a non-cubic grid, a surface impedance, a frequency change and the sampled rows of a larger
mesh; the solve against the oracle's dense LU (1e-4); state errors.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
TOL32 = 1e-5
TOL64 = 1e-9


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


@pytest.fixture(scope="module")
def l2(torch_cuda):
    """Level-2 icosphere (320 triangles, 480 RWG), 16^3 grid (plane-fused path), charge form on."""
    from synth import icosphere
    from oracle import operator as op, chargepot as cp
    from paper_2009_02281_gb300 import Context, EFIE
    xyz, tri = icosphere(2)
    grid = (16, 16, 16)
    ctx = Context(xyz, tri, grid, order=2, formulation=EFIE)
    ctx.set_charge_form(True)
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    ch = cp.setup_charge(prob)
    yield ctx, prob, ch
    ctx.close()


def test_setup_matches_oracle(l2):
    ctx, prob, ch = l2
    ex = ctx.export_charge()
    assert np.array_equal(ex["tanc"], ch["anc_t"])                        # anchors bit-exact
    got = sorted(zip(ex["rows"].tolist(), ex["cols"].tolist()))
    ref = sorted(zip(ch["rows"].tolist(), ch["cols"].tolist()))
    assert got == ref                                                     # near pattern bit-exact
    assert np.abs(ex["lp"] - ch["Lp"]).max() <= 1e-12 * np.abs(ch["Lp"]).max()
    # N_Pt on the same pairs (exported in internal row order: look the oracle value up per pair)
    key = {(r, c): v for r, c, v in zip(ch["rows"].tolist(), ch["cols"].tolist(), ch["NPt"])}
    ref_v = np.array([key[(r, c)] for r, c in zip(ex["rows"].tolist(), ex["cols"].tolist())])
    assert np.abs(ex["npt"] - ref_v).max() <= 1e-10 * np.abs(ref_v).max()


@pytest.mark.parametrize("nrhs", [1, 5, 37])
@pytest.mark.parametrize("path", [0, 1])
def test_product_matches_oracle(l2, torch_cuda, nrhs, path):
    torch = torch_cuda
    from synth import random_complex
    from oracle import chargepot as cp
    from paper_2009_02281_gb300 import F32
    ctx, prob, ch = l2
    ctx.set_path(path)
    assert ctx.matvec_path(F32) == path
    f = 1.3 * C0 / (2 * np.pi)
    x = random_complex((nrhs, ctx.nunk), seed=60 + nrhs)
    ref = np.stack([cp.matvec_efie_charge(prob, ch, f, xi) for xi in x])
    y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    ctx.set_path(0)
    assert _rel(y32, ref) <= TOL32
    for b in range(nrhs):
        assert _rel(y32[b], ref[b]) <= TOL32
    assert _rel(y64, ref) <= TOL64


def test_frequency_change_and_toggle(l2, torch_cuda):
    """Two frequencies in a row, then the RWG form again (the same context)."""
    torch = torch_cuda
    from synth import random_complex
    from oracle import chargepot as cp, operator as op
    ctx, prob, ch = l2
    x = random_complex((2, ctx.nunk), seed=70)
    xt = torch.tensor(x, dtype=torch.complex64, device="cuda")
    for kf in (0.4, 2.1):
        f = kf * C0 / (2 * np.pi)
        ref = np.stack([cp.matvec_efie_charge(prob, ch, f, xi) for xi in x])
        assert _rel(ctx.matvec(f, xt).cpu().numpy(), ref) <= TOL32
    ctx.set_charge_form(False)
    f = 2.1 * C0 / (2 * np.pi)
    ref = np.stack([op.matvec_efie(prob, f, xi) for xi in x])
    y = ctx.matvec(f, xt).cpu().numpy()
    ctx.set_charge_form(True)
    assert _rel(y, ref) <= TOL32


def test_divergence_free_current_has_no_scalar_potential(l2, torch_cuda):
    """A loop current (D x = 0): its scalar potential is exactly zero on both sides, so the
    comparison pins the vector-potential part of the charge-form product alone, at two
    frequencies whose k^-2 differ by a factor 9."""
    torch = torch_cuda
    from oracle import chargepot as cp
    ctx, prob, ch = l2
    D = ch["D"]
    # a divergence-free vector: projection of a random vector onto the null space of D
    rng = np.random.default_rng(3)
    v = rng.standard_normal(ctx.nunk) + 1j * rng.standard_normal(ctx.nunk)
    _, sv, vt = np.linalg.svd(D)
    null = vt[np.sum(sv > 1e-10 * sv[0]):]
    x = null.T @ (null.conj() @ v)
    assert np.linalg.norm(D @ x) <= 1e-12 * np.linalg.norm(x) * np.abs(D).max()
    for kf in (0.3, 0.9):
        f = kf * C0 / (2 * np.pi)
        ref = cp.matvec_efie_charge(prob, ch, f, x)
        y = ctx.matvec(f, torch.tensor(x[None], dtype=torch.complex128, device="cuda")).cpu().numpy()[0]
        assert _rel(y, ref) <= TOL64


def test_ragged_grid_and_surface_impedance(torch_cuda):
    """Non-cubic power-of-two grid (32 x 16 x 8) on a box, with a surface impedance (Gram term).
    Planes of unequal sides have no register-line kernels, so the charge form takes the generic
    path here in both precisions."""
    torch = torch_cuda
    from synth import box, random_complex
    from oracle import operator as op, chargepot as cp, sibc
    from paper_2009_02281_gb300 import Context, EFIE, F32
    xyz, tri = box([0, 0, 0], [4.0, 1.0, 0.5], [16, 4, 2])
    grid = (32, 16, 8)
    sigma = 5.8e7
    ctx = Context(xyz, tri, grid, order=2, formulation=EFIE, sigma=sigma)
    ctx.set_charge_form(True)
    assert ctx.matvec_path(F32) == 1
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    ch = cp.setup_charge(prob)
    f = 2.0 * C0 / (2 * np.pi)
    x = random_complex((3, ctx.nunk), seed=71)
    Gm = sibc.gram_dense(prob["rwg"])
    zs = sibc.surface_impedance(f, sigma)
    ref = np.stack([cp.matvec_efie_charge(prob, ch, f, xi) for xi in x]) + zs * (x @ Gm.T)
    y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    ctx.close()
    assert _rel(y32, ref) <= TOL32
    assert _rel(y64, ref) <= TOL64


def test_sampled_rows_larger_mesh(torch_cuda):
    """Level-4 icosphere (7680 unknowns) on a 32^3 grid, 64 RHS through the plane-fused path:
    sampled output rows against the oracle's row-restricted product."""
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op, chargepot as cp
    from paper_2009_02281_gb300 import Context, EFIE, F32
    xyz, tri = icosphere(4)
    grid = (32, 32, 32)
    ctx = Context(xyz, tri, grid, order=2, formulation=EFIE)
    ctx.set_charge_form(True)
    assert ctx.matvec_path(F32) == 0
    N = ctx.N
    rows = np.array([0, 1, N // 3, N // 2 + 5, N - 1])
    prob = op.setup(xyz, tri, 2, grid, radius=3, near_rows=rows)
    from oracle.rwg import rwg_arrays
    tris = np.unique(rwg_arrays(prob["rwg"])[0][rows].ravel())
    ch = cp.setup_charge(prob, tri_rows=tris)
    f = 4.0 * C0 / (2 * np.pi)
    B = 64
    x = random_complex((B, ctx.nunk), seed=72)
    y = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    ctx.close()
    for b in (0, B - 1):
        ref = cp.matvec_efie_charge(prob, ch, f, x[b], rows=rows)
        assert _rel(y[b, rows], ref) <= TOL32, b


def test_solve_matches_dense_lu(l2, torch_cuda):
    from synth import planewave_batch
    from oracle import chargepot as cp, solve as osolve, excitation
    ctx, prob, ch = l2
    k = 1.1
    f = k * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(2, seed=5)
    b = ctx.rhs_planewave(f, dirs, pols)
    tol = 1e-9
    x, stats, rc = ctx.solve(f, b, tol=tol, restart=80, max_iter=2000)
    assert rc == 0, stats
    Z = cp.dense_efie_charge(prob, ch, f)
    for w in range(2):
        VE, _ = excitation.planewave_rhs(prob["rwg"], k, dirs[w], pols[w])
        ref = osolve.lu_solve(Z, VE)
        assert _rel(x.cpu().numpy()[w], ref) <= 1e-4


def test_state_errors(torch_cuda):
    from synth import icosphere
    from paper_2009_02281_gb300 import AimxError, Context, EFIE, CFIE
    xyz, tri = icosphere(1)
    c = Context(xyz, tri, (8, 8, 8), formulation=CFIE)
    with pytest.raises(AimxError) as e:
        c.set_charge_form(True)
    assert e.value.code == -7
    c.close()
    c = Context(xyz, tri, (8, 8, 8), formulation=EFIE)
    with pytest.raises(AimxError) as e:
        c.export_charge()
    assert e.value.code == -7
    c.set_linear_term(True)
    with pytest.raises(AimxError) as e:
        c.set_charge_form(True)
    assert e.value.code == -7
    c.set_linear_term(False)
    c.set_charge_form(True)
    with pytest.raises(AimxError) as e:
        c.set_conventional_aim(True)
    assert e.value.code == -7
    c.close()


# ------------------------------------------------------------------ two-region (PMCHWT) charge form

@pytest.fixture(scope="module")
def l2p(torch_cuda):
    """Level-2 icosphere, eps_r = 4 inside, 16^3 grid (plane-fused path), two-region charge form."""
    from synth import icosphere
    from oracle import operator as op, chargepot as cp
    from paper_2009_02281_gb300 import Context, PMCHWT
    xyz, tri = icosphere(2)
    grid = (16, 16, 16)
    ctx = Context(xyz, tri, grid, order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    ctx.set_charge_form(True)
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    ch = cp.setup_charge(prob)
    yield ctx, prob, ch
    ctx.close()


@pytest.mark.parametrize("nrhs", [1, 5, 37])
@pytest.mark.parametrize("path", [0, 1])
def test_pmchwt_product_matches_oracle(l2p, torch_cuda, nrhs, path):
    """Both regions' scalar potentials in charge form, in the J and the M blocks, against
    ``matvec_pmchwt_charge``: plane-fused and generic paths, FP32 per RHS and FP64."""
    torch = torch_cuda
    from synth import random_complex
    from oracle import chargepot as cp
    from paper_2009_02281_gb300 import F32
    ctx, prob, ch = l2p
    ctx.set_path(path)
    assert ctx.matvec_path(F32) == path
    f = 1.1 * C0 / (2 * np.pi)
    x = random_complex((nrhs, ctx.nunk), seed=80 + nrhs)
    ref = np.stack([cp.matvec_pmchwt_charge(prob, ch, f, xi, 1.0, 4.0) for xi in x])
    y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    ctx.set_path(0)
    for b in range(nrhs):
        assert _rel(y32[b], ref[b]) <= TOL32, b
    assert _rel(y64, ref) <= TOL64


def test_pmchwt_solve_matches_dense_lu_and_sweep_refused(l2p, torch_cuda):
    """Plane-wave solve of the two-region charge form against the oracle's dense LU (1e-4);
    the batched sweep has no two-region charge product and says so."""
    from synth import planewave_batch
    from oracle import chargepot as cp, solve as osolve, excitation
    from oracle.constants import ETA0
    from paper_2009_02281_gb300 import AimxError
    ctx, prob, ch = l2p
    k = 0.9
    f = k * C0 / (2 * np.pi)
    dirs, pols = planewave_batch(1, seed=15)
    b = ctx.rhs_planewave(f, dirs, pols)
    x, stats, rc = ctx.solve(f, b, tol=1e-9, restart=100, max_iter=3000)
    assert rc == 0, stats
    Z = cp.dense_pmchwt_charge(prob, ch, f, 1.0, 4.0)
    VE, VH = excitation.planewave_rhs(prob["rwg"], k, dirs[0], pols[0], eta=ETA0)
    ref = osolve.lu_solve(Z, np.r_[VE, ETA0 * VH])
    assert _rel(x.cpu().numpy()[0], ref) <= 1e-4
    with pytest.raises(AimxError) as e:
        ctx.sweep_batched(np.array([f, 1.1 * f]), torch_cuda.stack([b, b]), tol=1e-6)
    assert e.value.code == -7


def test_pmchwt_sampled_rows_larger_mesh(torch_cuda):
    """Level-4 icosphere (15360 unknowns) on a 32^3 grid, 40 RHS through the plane-fused path:
    sampled rows of both blocks against the oracle's row-restricted two-region product."""
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op, chargepot as cp
    from oracle.rwg import rwg_arrays
    from paper_2009_02281_gb300 import Context, PMCHWT, F32
    xyz, tri = icosphere(4)
    grid = (32, 32, 32)
    ctx = Context(xyz, tri, grid, order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    ctx.set_charge_form(True)
    assert ctx.matvec_path(F32) == 0
    N = ctx.N
    rows = np.array([0, N // 3, N - 1])
    prob = op.setup(xyz, tri, 2, grid, radius=3, near_rows=rows)
    tris = np.unique(rwg_arrays(prob["rwg"])[0][rows].ravel())
    ch = cp.setup_charge(prob, tri_rows=tris)
    f = 3.0 * C0 / (2 * np.pi)
    B = 40
    x = random_complex((B, ctx.nunk), seed=81)
    y = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    ctx.close()
    for b in (0, B - 1):
        ref = cp.matvec_pmchwt_charge(prob, ch, f, x[b], 1.0, 4.0, rows=rows)
        assert _rel(np.r_[y[b, rows], y[b, N + rows]], ref) <= TOL32, b
