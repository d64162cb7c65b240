"""GPU parity of the AIMx setup and matvec against the FP64 oracle (through the C ABI).

Tolerances (stated by the method's accuracy targets): stencil anchors and the
near-region pattern bit-exact; rel-L2 <= 1e-9 for the FP64 matvec and <= 1e-5
for the FP32 matvec.  Weights and near values are FP64 on both sides and are
held to 1e-11 / 1e-10 of their scale.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
TOL64 = 1e-9
TOL32 = 1e-5


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


def _mesh(level):
    from synth import icosphere
    return icosphere(level)


@pytest.fixture(scope="module")
def efie_l2(torch_cuda):
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE
    xyz, tri = _mesh(2)
    ctx = Context(xyz, tri, (12, 12, 12), order=2, formulation=EFIE)
    prob = op.setup(xyz, tri, 2, (12, 12, 12), radius=3)
    yield ctx, prob
    ctx.close()


@pytest.fixture(scope="module")
def pmchwt_l1(torch_cuda):
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, PMCHWT
    xyz, tri = _mesh(1)
    ctx = Context(xyz, tri, (8, 8, 8), order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    prob = op.setup(xyz, tri, 2, (8, 8, 8), radius=3)
    yield ctx, prob
    ctx.close()


def test_setup_parity(efie_l2):
    ctx, prob = efie_l2
    ex = ctx.export_setup()
    assert np.array_equal(ex["anchors"], prob["anc"])                 # bit-exact
    assert np.array_equal(ex["row_ptr"], prob["row_ptr"])             # bit-exact pattern
    assert np.array_equal(ex["cols"], prob["cols"])
    lam = prob["lam"]
    assert np.abs(ex["weights"] - lam).max() <= 1e-11 * np.abs(lam).max()
    for k in ("NA", "NP", "NK"):
        ref = prob["near"][k]
        assert np.abs(ex[k] - ref).max() <= 1e-10 * np.abs(ref).max(), k
    g = ctx.info
    assert np.allclose(g["grid_h"], prob["grid"]["h"], rtol=0, atol=0)
    assert np.allclose(g["grid_origin"], prob["grid"]["origin"], rtol=0, atol=0)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_efie_matvec_parity(efie_l2, torch_cuda, nrhs):
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    ctx, prob = efie_l2
    freq = 1.3 * C0 / (2 * np.pi)
    x = random_complex((nrhs, ctx.nunk), seed=11 + nrhs)
    ref = np.stack([op.matvec_efie(prob, freq, xi) for xi in x])
    y64 = ctx.matvec(freq, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    y32 = ctx.matvec(freq, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert _relerr(y64, ref) <= TOL64
    assert _relerr(y32, ref) <= TOL32
    for b in range(nrhs):
        assert _relerr(y32[b], ref[b]) <= TOL32


def test_pmchwt_matvec_parity(pmchwt_l1, torch_cuda):
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    ctx, prob = pmchwt_l1
    freq = 0.9 * C0 / (2 * np.pi)
    x = random_complex((2, ctx.nunk), seed=7)
    ref = np.stack([op.matvec_pmchwt(prob, freq, xi, 1.0, 4.0) for xi in x])
    y64 = ctx.matvec(freq, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    y32 = ctx.matvec(freq, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert _relerr(y64, ref) <= TOL64
    assert _relerr(y32, ref) <= TOL32
    ex = ctx.export_setup()
    assert np.abs(ex["NK"] - prob["near"]["NK"]).max() <= 1e-10 * np.abs(prob["near"]["NK"]).max()


def test_frequency_cache_switch(efie_l2, torch_cuda):
    """Products at two frequencies in turn reuse the static data and regenerate H(k)."""
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    ctx, prob = efie_l2
    x = random_complex((1, ctx.nunk), seed=3)
    xt = torch.tensor(x, dtype=torch.complex128, device="cuda")
    for k in (0.7, 2.1, 0.7):
        f = k * C0 / (2 * np.pi)
        ref = op.matvec_efie(prob, f, x[0])
        assert _relerr(ctx.matvec(f, xt).cpu().numpy()[0], ref) <= TOL64


def test_matvec_deterministic(efie_l2, torch_cuda):
    torch = torch_cuda
    from synth import random_complex
    ctx, _ = efie_l2
    x = torch.tensor(random_complex((4, ctx.nunk), seed=5), dtype=torch.complex64, device="cuda")
    f = 1.1 * C0 / (2 * np.pi)
    a = ctx.matvec(f, x).cpu().numpy()
    b = ctx.matvec(f, x).cpu().numpy()
    assert np.array_equal(a.view(np.float32), b.view(np.float32))


def test_matvec_host_path(efie_l2, torch_cuda):
    torch = torch_cuda
    from synth import random_complex
    ctx, _ = efie_l2
    x = random_complex((2, ctx.nunk), seed=9)
    f = 1.1 * C0 / (2 * np.pi)
    yd = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    yh = ctx.matvec_host(f, x)
    assert np.array_equal(yd, yh)


def test_setup_errors(torch_cuda):
    from paper_2009_02281_gb300 import Context, AimxError
    xyz, tri = _mesh(1)
    with pytest.raises(AimxError) as e:
        Context(xyz, tri, (8, 8, 8), h=(0.3, 0.3, 0.3), origin=(0.0, 0.0, 0.0))
    assert e.value.code == -3
    bad = tri.copy()
    bad[0] = bad[0][[0, 2, 1]]
    with pytest.raises(AimxError) as e:
        Context(xyz, bad, (8, 8, 8))
    assert e.value.code == -2


def test_config1_sized_efie(torch_cuda):
    """1920-unknown PEC sphere on a 24^3 grid (padded to 48^3 = 3 * 16 per axis), every row checked."""
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE
    xyz, tri = icosphere(3)
    freq = C0 / 2.0                                 # diameter = 1 wavelength
    ctx = Context(xyz, tri, (24, 24, 24), order=2, formulation=EFIE)
    prob = op.setup(xyz, tri, 2, (24, 24, 24), radius=3)
    x = random_complex((1, ctx.nunk), seed=21)
    ref = op.matvec_efie(prob, freq, x[0])
    y64 = ctx.matvec(freq, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()[0]
    y32 = ctx.matvec(freq, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()[0]
    ctx.close()
    assert _relerr(y64, ref) <= TOL64
    assert _relerr(y32, ref) <= TOL32


@pytest.mark.parametrize("form", ["efie", "pmchwt"])
def test_cufft_comparison_path_parity(efie_l2, pmchwt_l1, torch_cuda, form):
    """The plain comparison path (cuFFT transforms of the full padded grids) computes the same product."""
    torch = torch_cuda
    from synth import random_complex
    from oracle import operator as op
    ctx, prob = efie_l2 if form == "efie" else pmchwt_l1
    f = 1.1 * C0 / (2 * np.pi)
    x = random_complex((2, ctx.nunk), seed=61)
    if form == "efie":
        ref = np.stack([op.matvec_efie(prob, f, v) for v in x])
    else:
        ref = np.stack([op.matvec_pmchwt(prob, f, v, 1.0, 4.0) for v in x])
    ctx.set_path(2)
    try:
        assert ctx.matvec_path() == 2
        y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
        y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    finally:
        ctx.set_path(0)
    assert _relerr(y64, ref) <= TOL64
    assert _relerr(y32, ref) <= TOL32


@pytest.mark.parametrize("form", ["efie", "pmchwt"])
def test_mixed_radix_pads(torch_cuda, form):
    """FFT lengths 3 * 2^k: the default pad of a 12^3 grid is 24 per axis (radix 3 then radix 2);
    explicit pads mixing 24, 32 and 48 per axis, and the power-of-two pad, give the oracle's
    product (it sums over the grid directly and has no pad) in FP64 and FP32."""
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE, PMCHWT
    xyz, tri = icosphere(2)
    grid = (12, 12, 12)
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    f = 1.3 * C0 / (2 * np.pi)
    fm = EFIE if form == "efie" else PMCHWT
    ref = None
    for pad in (None, (24, 32, 48), (32, 32, 32), (48, 24, 24)):
        ctx = Context(xyz, tri, grid, order=2, formulation=fm, eps_out=1.0, eps_in=4.0, pad=pad)
        assert ctx.info["pad"] == (pad or (24, 24, 24))
        x = random_complex((2, ctx.nunk), seed=91)
        if ref is None:
            if form == "efie":
                ref = np.stack([op.matvec_efie(prob, f, xi) for xi in x])
            else:
                ref = np.stack([op.matvec_pmchwt(prob, f, xi, 1.0, 4.0) for xi in x])
        y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
        y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
        ctx.close()
        assert np.linalg.norm(y64 - ref) / np.linalg.norm(ref) <= 1e-9, pad
        assert np.linalg.norm(y32 - ref) / np.linalg.norm(ref) <= 1e-5, pad


@pytest.mark.parametrize("grid,pad,nrhs", [((12, 12, 12), (24, 24, 24), 16), ((12, 12, 12), (32, 32, 32), 8),
                                           ((12, 12, 12), (48, 48, 48), 4), ((8, 8, 8), (16, 16, 16), 32),
                                           ((12, 12, 12), (64, 64, 64), 2)])
def test_register_line_ffts(torch_cuda, grid, pad, nrhs):
    """The generic path's register-line FFTs (one line per thread): FP32 lines of 16 to 64 points
    always, FP64 lines of 16 to 48 points when a transform has at least 32768 z lines, which the
    right-hand-side counts here reach (64 points: FP32 only).  The batched FP64 product must equal
    the same product taken one RHS at a time (shared-memory line FFTs) to rounding, and both
    precisions must match the oracle on the first and last RHS."""
    torch = torch_cuda
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, grid, order=2, formulation=EFIE, pad=pad)
    ctx.set_path(1)
    f = 1.1 * C0 / (2 * np.pi)
    x = random_complex((nrhs, ctx.nunk), seed=93)
    x64 = torch.tensor(x, dtype=torch.complex128, device="cuda")
    y64 = ctx.matvec(f, x64).cpu().numpy()
    one = np.stack([ctx.matvec(f, x64[b:b + 1]).cpu().numpy()[0] for b in range(nrhs)])
    y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
    ctx.close()
    assert np.linalg.norm(y64 - one) / np.linalg.norm(one) <= 1e-12
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    for b in (0, nrhs - 1):
        ref = op.matvec_efie(prob, f, x[b])
        assert np.linalg.norm(y64[b] - ref) / np.linalg.norm(ref) <= 1e-9
        assert np.linalg.norm(y32[b] - ref) / np.linalg.norm(ref) <= 1e-5
