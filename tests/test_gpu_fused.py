"""GPU parity of the plane-fused FP32 matvec (grids padded to exactly 2N per axis).

Checks the fused path against the FP64 oracle (rel-L2 <= 1e-5), against the
generic path of the same library, and at the full 61440-unknown dielectric
sphere workload on sampled rows the oracle computes by direct summation, in
the batch size and launch configuration the benchmark times.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
TOL32 = 1e-5
TOL64 = 1e-9


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


@pytest.mark.parametrize("form", ["efie", "pmchwt"])
@pytest.mark.parametrize("nrhs", [1, 5, 9, 37])
def test_fused_matches_oracle_and_generic(torch_cuda, form, nrhs):
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE, PMCHWT, F32
    xyz, tri = icosphere(2)
    grid = (16, 16, 16)
    fm = EFIE if form == "efie" else PMCHWT
    ctx = Context(xyz, tri, grid, order=2, formulation=fm, eps_out=1.0, eps_in=4.0)
    assert ctx.matvec_path(F32) == 0, "16^3 grid padded to 32^3 must take the plane-fused path"
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    freq = 1.4 * C0 / (2 * np.pi)
    x = random_complex((nrhs, ctx.nunk), seed=31 + nrhs)
    if form == "efie":
        ref = np.stack([op.matvec_efie(prob, freq, xi) for xi in x])
    else:
        ref = np.stack([op.matvec_pmchwt(prob, freq, xi, 1.0, 4.0) for xi in x])
    xt = torch.tensor(x, dtype=torch.complex64, device="cuda")
    yf = ctx.matvec(freq, xt).cpu().numpy()
    ctx.set_path(1)
    yg = ctx.matvec(freq, xt).cpu().numpy()
    ctx.set_path(0)
    ctx.close()
    assert _relerr(yf, ref) <= TOL32
    for b in range(nrhs):
        assert _relerr(yf[b], ref[b]) <= TOL32
    assert _relerr(yf, yg) <= TOL32


def test_fused_ragged_grid(torch_cuda):
    """Non-cubic power-of-two grid (32 x 16 x 8) on a box-like mesh spanning several tiles."""
    torch = torch_cuda
    from synth import box, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE, F32
    xyz, tri = box([0, 0, 0], [4.0, 1.0, 0.5], [16, 4, 2])
    grid = (32, 16, 8)
    ctx = Context(xyz, tri, grid, order=2, formulation=EFIE)
    assert ctx.matvec_path(F32) == 0
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    freq = 2.0 * C0 / (2 * np.pi)
    x = random_complex((3, ctx.nunk), seed=2)
    ref = np.stack([op.matvec_efie(prob, freq, xi) for xi in x])
    y = ctx.matvec(freq, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    ctx.close()
    assert _relerr(y, ref) <= TOL32


def test_fused_deterministic(torch_cuda):
    torch = torch_cuda
    from synth import icosphere, random_complex
    from paper_2009_02281_gb300 import Context, PMCHWT
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (16, 16, 16), formulation=PMCHWT, eps_in=3.0)
    x = torch.tensor(random_complex((6, ctx.nunk), seed=8), dtype=torch.complex64, device="cuda")
    f = 1.0 * C0 / (2 * np.pi)
    a = ctx.matvec(f, x).cpu().numpy()
    b = ctx.matvec(f, x).cpu().numpy()
    ctx.close()
    assert np.array_equal(a.view(np.float32), b.view(np.float32))


@pytest.mark.parametrize("form,order", [("pmchwt", 2), ("efie", 1), ("efie", 3)])
def test_fused_planes_beyond_shared_memory(torch_cuda, form, order):
    """A grid plane with more bases than the inverse-xy kernel keeps in shared memory sums its
    interpolation partials in the output array (forced here with a cap of 8 bases per plane):
    bitwise the product of the shared-memory form, and the oracle's within the FP32 tolerance.
    Orders 1 and 3 take the two-bases-per-iteration loop, order 2 the four-bases one."""
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE, PMCHWT, F32
    xyz, tri = icosphere(2)
    grid = (16, 16, 16)
    fm = EFIE if form == "efie" else PMCHWT
    ctx = Context(xyz, tri, grid, order=order, formulation=fm, eps_out=1.0, eps_in=4.0)
    assert ctx.matvec_path(F32) == 0
    f = 1.2 * C0 / (2 * np.pi)
    x = random_complex((3, ctx.nunk), seed=77)
    xt = torch.tensor(x, dtype=torch.complex64, device="cuda")
    a = ctx.matvec(f, xt).cpu().numpy()
    ctx.set_plane_cap(8)
    b = ctx.matvec(f, xt).cpu().numpy()
    ctx.set_plane_cap(0)
    c = ctx.matvec(f, xt).cpu().numpy()
    ctx.close()
    assert np.array_equal(a.view(np.float32), b.view(np.float32))
    assert np.array_equal(a.view(np.float32), c.view(np.float32))
    prob = op.setup(xyz, tri, order, grid, radius=3)
    if form == "efie":
        ref = np.stack([op.matvec_efie(prob, f, xi) for xi in x])
    else:
        ref = np.stack([op.matvec_pmchwt(prob, f, xi, 1.0, 4.0) for xi in x])
    assert _relerr(b, ref) <= TOL32


@pytest.fixture(scope="module")
def full_workload(torch_cuda):
    """The benchmark workload: 61440 unknowns, 64^3 grid padded to 128^3, 64 RHS."""
    from synth import workloads
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, PMCHWT
    wl = workloads.dielectric_sphere_61440()
    ctx = Context(wl["xyz"], wl["tri"], wl["grid_n"], order=wl["order"], formulation=PMCHWT,
                  eps_out=wl["eps_out"], eps_in=wl["eps_in"], near_radius=wl["radius"])
    N = ctx.N
    rows = np.array([0, 1, N // 3, N // 2 + 7, N - 1])
    prob = op.setup(wl["xyz"], wl["tri"], wl["order"], wl["grid_n"], radius=wl["radius"], near_rows=rows)
    yield wl, ctx, prob, rows
    ctx.close()


def test_full_workload_sampled_rows(full_workload, torch_cuda):
    """Bench launch configuration (64 RHS, FP32, plane-fused); rows checked against direct summation."""
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import F32
    wl, ctx, prob, rows = full_workload
    assert ctx.matvec_path(F32) == 0
    B = wl["nrhs"]
    x = random_complex((B, ctx.nunk), seed=77)
    y = ctx.matvec(wl["freq"], torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    N = ctx.N
    for b in (0, B - 1):
        ref = op.matvec_pmchwt(prob, wl["freq"], x[b], wl["eps_out"], wl["eps_in"], rows=rows)
        got = np.r_[y[b, rows], y[b, N + rows]]
        assert _relerr(got, ref) <= TOL32, b


def test_full_workload_fp64_sampled_rows(full_workload, torch_cuda):
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    wl, ctx, prob, rows = full_workload
    x = random_complex((1, ctx.nunk), seed=78)
    y = ctx.matvec(wl["freq"], torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()[0]
    ref = op.matvec_pmchwt(prob, wl["freq"], x[0], wl["eps_out"], wl["eps_in"], rows=rows)
    N = ctx.N
    assert _relerr(np.r_[y[rows], y[N + rows]], ref) <= TOL64


def test_full_workload_reciprocity(full_workload, torch_cuda):
    """Any-size property: diag(1,-1) A is complex symmetric, so u^T D A v = v^T D A u."""
    torch = torch_cuda
    from synth import random_complex
    wl, ctx, prob, rows = full_workload
    N = ctx.N
    uv = random_complex((2, ctx.nunk), seed=90)
    y = ctx.matvec(wl["freq"], torch.tensor(uv, dtype=torch.complex128, device="cuda")).cpu().numpy()
    D = np.r_[np.ones(N), -np.ones(N)]
    a = np.sum(uv[0] * D * y[1])
    b = np.sum(uv[1] * D * y[0])
    # near-matrix symmetry is limited by the outer quadrature of touching triangle pairs
    assert abs(a - b) <= 2e-3 * max(abs(a), abs(b))
