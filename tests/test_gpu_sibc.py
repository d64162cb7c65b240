"""GPU parity of the surface impedance term, delta-gap ports and Y-parameter sweeps.

Two gap-dipole copper bars in a dielectric background: the EFIE + Z_s G
product (FP64 generic path 1e-9, FP32 paths 1e-5) against the oracle's direct
summation, the port vectors against the oracle's gap-edge search (exact), and
the Y-parameters of a swept solve against the oracle's dense LU (1e-4).  The
bars are millimetre-sized so that the swept frequencies put them near half a
wavelength: at k L << 1 the plain EFIE is too ill-conditioned for GMRES with
the diagonal preconditioner (the low-frequency breakdown the AEFIE addresses).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIGMA = 5.8e7
EPS = 3.5
L, W, T = 6e-3, 1e-3, 0.5e-3
GRID = (16, 8, 8)


@pytest.fixture(scope="module")
def bars():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02281_gb300 import build, Context, EFIE, Port
    from synth import box, merge_meshes
    from oracle import operator as op
    build.build()
    parts = [box([0, 2 * W * i, 0], [L, 2 * W * i + W, T], [6, 2, 2]) for i in range(2)]
    xyz, tri, _ = merge_meshes(parts)
    ctx = Context(xyz, tri, GRID, order=2, formulation=EFIE, eps_out=EPS, sigma=SIGMA)
    prob = op.setup(xyz, tri, 2, GRID, radius=3)
    ports_o = [([L / 2, 0, 0], [1, 0, 0], [-1, 2 * W * i - 1e-6, -1], [1, 2 * W * i + W + 1e-6, 1]) for i in range(2)]
    ports = [Port.make(*p) for p in ports_o]
    yield torch, ctx, prob, ports, ports_o
    ctx.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_sibc_product_parity(bars):
    torch, ctx, prob, _, _ = bars
    from synth import random_complex
    from oracle import sibc
    f = 2e10
    x = random_complex((2, ctx.nunk), seed=3)
    ref = np.stack([sibc.matvec_efie_sibc(prob, f, v, SIGMA, EPS) for v in x])
    y64 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert _rel(y64, ref) <= 1e-9
    for path in (0, 1):
        ctx.set_path(path)
        y32 = ctx.matvec(f, torch.tensor(x, dtype=torch.complex64, device="cuda")).cpu().numpy()
        assert _rel(y32, ref) <= 1e-5, path
    ctx.set_path(0)


def test_port_vectors_match_oracle(bars):
    torch, ctx, prob, ports, ports_o = bars
    from oracle import sibc
    c, ne = ctx.port_vectors(ports)
    for p in range(2):
        ref = sibc.port_vector(prob["rwg"], ports_o[p])
        assert np.allclose(c[p], ref, rtol=1e-12, atol=0)
        assert ne[p] == np.count_nonzero(ref)


def test_y_parameters_match_dense_lu(bars):
    torch, ctx, prob, ports, ports_o = bars
    from oracle import sibc
    from paper_2009_02281_gb300 import F64, PRECOND_BLOCK
    freqs = [1.2e10, 2.0e10]
    # restart above the 336 unknowns: full GMRES, which ends within n iterations
    Y, stats, rc = ctx.sweep_ports(freqs, ports, tol=1e-10, restart=400, max_iter=3000, inner_precision=F64)
    assert rc == 0, stats
    for k, f in enumerate(freqs):
        ref = sibc.y_parameters(sibc.dense_efie_sibc(prob, f, SIGMA, EPS), prob["rwg"], ports_o)
        assert _rel(Y[k], ref) <= 1e-4, (f, Y[k], ref)
    # the block preconditioner includes the surface-impedance term and reaches the same answer
    Yb, _, rcb = ctx.sweep_ports(freqs[:1], ports, tol=1e-10, restart=400, max_iter=3000, inner_precision=F64,
                                 precond=PRECOND_BLOCK)
    assert rcb == 0
    assert _rel(Yb[0], Y[0]) <= 1e-6
