"""GPU parity of the linear-term modification (Sec. III-A-3, Eqs. linterm and Lmatdecomplin).

The overlap pattern is compared exactly and its FP64 values to 1e-10 of their
scale (both sides integrate the same closed forms with the same 5 x 5 rule);
products with the term on are held to the matvec tolerances (FP64 1e-9, FP32
1e-5) against the oracle's product, on both FP32 paths, EFIE and PMCHWT.
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


@pytest.fixture(scope="module")
def efie(torch_cuda):
    from synth import icosphere
    from oracle import operator as op, linterm
    from paper_2009_02281_gb300 import Context, EFIE
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (12, 12, 12), order=2, formulation=EFIE)
    prob = op.setup(xyz, tri, 2, (12, 12, 12), radius=3)
    yield ctx, prob, linterm.lin_matrices(prob)
    ctx.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _to_csr(rows, cols, vals, N):
    order = np.lexsort((cols, rows))
    rp = np.zeros(N + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols[order], [v[order] for v in vals]


def test_state_errors(efie):
    from paper_2009_02281_gb300 import AimxError
    from synth import icosphere
    from paper_2009_02281_gb300 import Context, EFIE
    xyz, tri = icosphere(1)
    c = Context(xyz, tri, (8, 8, 8), formulation=EFIE)
    with pytest.raises(AimxError) as e:
        c.export_linear_term()
    assert e.value.code == -7
    with pytest.raises(AimxError) as e:
        c._check(c._lib.aimx_set_linear_term(c._ctx, 2))
    assert e.value.code == -1
    c.close()


def test_values_match_oracle(efie):
    ctx, prob, (rows, cols, NA, NP) = efie
    ctx.set_linear_term(True)
    ex = ctx.export_linear_term()
    rp, cs, (na, npv) = _to_csr(rows, cols, (NA, NP), prob["N"])
    assert np.array_equal(ex["row_ptr"], rp)
    assert np.array_equal(ex["cols"], cs)
    assert np.abs(ex["NA"] - na).max() <= 1e-10 * np.abs(na).max()
    assert np.abs(ex["NP"] - npv).max() <= 1e-10 * np.abs(npv).max()


@pytest.mark.parametrize("nrhs", [1, 3])
def test_efie_product_parity(efie, torch_cuda, nrhs):
    torch = torch_cuda
    from synth import random_complex
    from oracle import linterm
    ctx, prob, lin = efie
    ctx.set_linear_term(True)
    f = 0.3 * C0
    x = random_complex((nrhs, ctx.nunk), seed=30 + nrhs)
    ref = np.stack([linterm.matvec_efie_lin(prob, f, v, lin=lin) for v in x])
    y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert _rel(y64, ref) <= 1e-9
    for path in (0, 1):
        ctx.set_path(path)
        y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
        assert _rel(y32, ref) <= 1e-5, path
    ctx.set_path(0)


def test_toggle_restores_unmodified_product(efie, torch_cuda):
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    ctx, prob, _ = efie
    f = 0.25 * C0
    x = torch.tensor(random_complex((2, ctx.nunk), seed=8), dtype=torch.complex64, device="cuda")
    ctx.set_linear_term(True)
    on = ctx.matvec(f, x).cpu().numpy()
    ctx.set_linear_term(False)
    off = ctx.matvec(f, x).cpu().numpy()
    ref = np.stack([op.matvec_efie(prob, f, v) for v in x.cpu().numpy().astype(np.complex128)])
    assert _rel(off, ref) <= 1e-5
    assert _rel(on, off) > 1e-4            # the term changes the product at this frequency


def test_pmchwt_product_parity(torch_cuda):
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op, linterm
    from paper_2009_02281_gb300 import Context, PMCHWT
    xyz, tri = icosphere(1)
    ctx = Context(xyz, tri, (8, 8, 8), order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    prob = op.setup(xyz, tri, 2, (8, 8, 8), radius=3)
    ctx.set_linear_term(True)
    f = 0.9 * C0 / (2 * np.pi)
    x = random_complex((2, ctx.nunk), seed=12)
    ref = np.stack([linterm.matvec_pmchwt_lin(prob, f, v, 1.0, 4.0) for v in x])
    y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert _rel(y64, ref) <= 1e-9
    for path in (0, 1):
        ctx.set_path(path)
        y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
        assert _rel(y32, ref) <= 1e-5, path
    ctx.close()


def test_solve_matches_dense_solution(efie, torch_cuda):
    """GMRES with the term on converges to the dense oracle's solution of the modified system."""
    torch = torch_cuda
    from synth import random_complex
    from oracle import linterm
    from paper_2009_02281_gb300 import F64
    ctx, prob, lin = efie
    ctx.set_linear_term(True)
    f = 0.3 * C0
    b = random_complex((1, ctx.nunk), seed=77)
    Z = linterm.dense_efie_lin(prob, f, lin=lin)
    xr = np.linalg.solve(Z, b[0])
    # restart above the 480 unknowns: full GMRES
    x, stats, rc = ctx.solve(f, torch.tensor(b, dtype=torch.complex128, device="cuda"), tol=1e-10,
                             restart=500, max_iter=2000, inner_precision=F64)
    assert rc == 0, stats
    xg = x.cpu().numpy()[0]
    assert np.linalg.norm(Z @ xg - b[0]) <= 1e-8 * np.linalg.norm(b[0])
    assert _rel(xg, xr) <= 1e-6


def test_batch_recaptures_after_toggle(torch_cuda):
    torch = torch_cuda
    from synth import icosphere, random_complex
    from paper_2009_02281_gb300 import Batch, Context, EFIE
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (12, 12, 12), formulation=EFIE)
    f = 0.3 * C0
    x = torch.tensor(random_complex((2, ctx.nunk), seed=5), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    batch = Batch([ctx])
    batch.matvec([f], [x], [y])
    torch.cuda.synchronize()
    off = y.cpu().numpy()
    ctx.set_linear_term(True)
    batch.matvec([f], [x], [y])
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), ctx.matvec(f, x).cpu().numpy())
    assert not np.array_equal(y.cpu().numpy(), off)
    batch.close()
    ctx.close()
