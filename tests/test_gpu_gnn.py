"""GPU parity of the learned near-field preconditioner (network, loss, gradients, apply).

The CUDA network runs with BF16-rounded parameters and FP32 activations; the
oracle (oracle/gnn.py, float64) is given the same BF16-rounded parameters, its
own float64 features and D^{-1}, and probe pairs y = A z formed with its dense
AIMx matrix.  Tolerances: features and bases 1e-5 (FP32 storage of FP64 values), network
outputs and the loss 1e-4 relative, parameter gradients 2e-3 relative per
parameter block (FP32 accumulation over every near edge; a ReLU whose
pre-activation sits within FP32 rounding of zero may switch), the
preconditioner application 1e-5 relative.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS_IN = 4.0


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02281_gb300 import build
    build.build()
    return torch


def _bf16(a):
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _params(K, seed, layers=4):
    from oracle import gnn
    rng = np.random.default_rng(seed)
    p = gnn.init_params(seed, layers=layers, K=K)
    for k in ("E", "G"):
        p[k] = 0.05 * rng.standard_normal(p[k].shape)
    for k in ("f", "g", "u"):
        p[k] = 0.02 * rng.standard_normal(p[k].shape)
    for l in range(1, layers + 1):
        p[f"c{l}"] = 0.1 * rng.standard_normal(p[f"c{l}"].shape)
        p[f"d{l}"] = 0.1 * rng.standard_normal(p[f"d{l}"].shape)
    flat = np.concatenate([p[k].ravel() for k in gnn.PARAM_ORDER if k in p]).astype(np.float32)
    rounded = _bf16(flat)
    out, off = {}, 0
    for k in gnn.PARAM_ORDER:
        if k not in p:
            continue
        n = p[k].size
        out[k] = rounded[off:off + n].astype(np.float64).reshape(p[k].shape)
        off += n
    return flat, out


def _case(form):
    from synth import icosphere
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE, PMCHWT
    xyz, tri = icosphere(1)
    prob = op.setup(xyz, tri, 2, (8, 8, 8), radius=3)
    if form == "efie":
        ctx = Context(xyz, tri, (8, 8, 8), order=2, formulation=EFIE)
    else:
        ctx = Context(xyz, tri, (8, 8, 8), order=2, formulation=PMCHWT, eps_out=1.0, eps_in=EPS_IN)
    return ctx, prob


@pytest.fixture(scope="module", params=["efie", "pmchwt"])
def case(request, torch_cuda):
    ctx, prob = _case(request.param)
    yield request.param, ctx, prob
    ctx.close()


FREQ = 2.5e8


def _oracle_inputs(form, prob):
    from oracle import gnn
    kw = {} if form == "efie" else dict(eps_out=1.0, eps_in=EPS_IN)
    x, e, basis, rows, cols = gnn.features(prob, FREQ, **kw)
    dinv = gnn.diag_inverse(prob, FREQ, **kw)
    return x, e, basis, rows, cols, dinv


def _edge_map(ctx_rows, ctx_cols, rows, cols):
    pos = {(int(m), int(n)): i for i, (m, n) in enumerate(zip(rows, cols))}
    return np.array([pos[(int(m), int(n))] for m, n in zip(ctx_rows, ctx_cols)])


def test_features_parity(case):
    form, ctx, prob = case
    x, e, basis, rows, cols, _ = _oracle_inputs(form, prob)
    node, edge, bas, r, c = ctx.gnn_features(FREQ)
    assert len(r) == len(rows)
    idx = _edge_map(r, c, rows, cols)
    assert np.allclose(node, x, rtol=1e-5, atol=1e-6)
    assert np.allclose(edge, e[idx], rtol=1e-5, atol=1e-6)
    assert np.allclose(bas, basis[idx], rtol=1e-5, atol=1e-6)


def test_forward_parity(case):
    from oracle import gnn
    from paper_2009_02281_gb300 import Gnn, EFIE, PMCHWT
    form, ctx, prob = case
    K = 2 if form == "efie" else 8
    flat, p = _params(K, 11)
    x, e, basis, rows, cols, _ = _oracle_inputs(form, prob)
    o_ref, g_ref, _ = gnn.forward(p, x, e, basis, rows, cols)
    net = Gnn(EFIE if K == 2 else PMCHWT)
    net.set_params(flat)
    o, g = ctx.gnn_outputs(net, FREQ)
    _, _, _, r, c = ctx.gnn_features(FREQ)
    idx = _edge_map(r, c, rows, cols)
    so = np.abs(o_ref).max()
    assert np.abs(o - o_ref[idx]).max() <= 1e-4 * so
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    net.close()


def _probes(form, prob, P, seed):
    from oracle import operator as op
    rng = np.random.default_rng(seed)
    if form == "efie":
        A = op.dense_efie(prob, FREQ)
    else:
        A = op.dense_pmchwt(prob, FREQ, 1.0, EPS_IN)
    n = A.shape[0]
    Z = (rng.standard_normal((P, n)) + 1j * rng.standard_normal((P, n))).astype(np.complex64)
    Y = (Z.astype(np.complex128) @ A.T).astype(np.complex64)
    return Z, Y


def test_loss_and_gradient_parity(case, torch_cuda):
    torch = torch_cuda
    from oracle import gnn
    from paper_2009_02281_gb300 import Gnn, EFIE, PMCHWT
    form, ctx, prob = case
    K = 2 if form == "efie" else 8
    flat, p = _params(K, 5)
    x, e, basis, rows, cols, dinv = _oracle_inputs(form, prob)
    Z, Y = _probes(form, prob, 4, 9)
    L_ref, G_ref = gnn.loss_and_grads(p, x, e, basis, rows, cols, dinv, Y.astype(np.complex128),
                                      Z.astype(np.complex128), K)
    net = Gnn(EFIE if K == 2 else PMCHWT)
    net.set_params(flat)
    Zd = torch.from_numpy(Z).cuda()
    Yd = torch.from_numpy(Y).cuda()
    L, g = net.loss_grad(ctx, FREQ, Zd, Yd)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    off = 0
    for k in gnn.PARAM_ORDER:
        n = G_ref[k].size
        ref = G_ref[k].ravel()
        got = g[off:off + n]
        off += n
        scale = max(np.linalg.norm(ref), 1e-6 * abs(L_ref))
        assert np.linalg.norm(got - ref) <= 2e-3 * scale, k
    assert off == net.n_params
    # deterministic: a second evaluation is bitwise identical
    L2, g2 = net.loss_grad(ctx, FREQ, Zd, Yd)
    assert L2 == L and np.array_equal(g2, g)
    net.close()


def test_learned_apply_parity(case, torch_cuda):
    torch = torch_cuda
    from oracle import gnn
    from paper_2009_02281_gb300 import Gnn, EFIE, PMCHWT, PRECOND_LEARNED
    form, ctx, prob = case
    K = 2 if form == "efie" else 8
    flat, p = _params(K, 3)
    x, e, basis, rows, cols, dinv = _oracle_inputs(form, prob)
    o, g, _ = gnn.forward(p, x, e, basis, rows, cols)
    oc, gc = gnn.to_complex_blocks(o, g, K)
    net = Gnn(EFIE if K == 2 else PMCHWT)
    net.set_params(flat)
    ctx.gnn_attach(net)
    net.close()  # the context keeps its own copy
    rng = np.random.default_rng(2)
    n = ctx.nunk
    V = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    z = ctx.precond_apply(FREQ, torch.from_numpy(V).cuda(), precond=PRECOND_LEARNED).cpu().numpy()
    for b in range(3):
        ref = gnn.apply_precond(dinv, oc, gc, rows, cols, V[b], K)
        assert np.linalg.norm(z[b] - ref) <= 1e-5 * np.linalg.norm(ref)
    ctx.gnn_attach(None)


def test_errors(torch_cuda):
    from paper_2009_02281_gb300 import Gnn, PMCHWT, AimxError, PRECOND_LEARNED
    torch = torch_cuda
    ctx, prob = _case("efie")
    net = Gnn(PMCHWT)
    with pytest.raises(AimxError) as ei:
        ctx.gnn_attach(net)
    assert ei.value.code == -1
    b = torch.ones((1, ctx.nunk), dtype=torch.complex128, device="cuda")
    with pytest.raises(AimxError) as ei:
        ctx.solve(FREQ, b, precond=PRECOND_LEARNED)
    assert ei.value.code == -7
    net.close()
    ctx.close()


def test_training_lowers_loss_and_learned_solve_matches_lu(torch_cuda):
    """Adam steps on one EFIE sphere at ka = pi: the probe loss falls, the learned
    preconditioner needs fewer GMRES iterations than the diagonal one, and the solve
    reaches the dense-LU solution of the same AIMx system."""
    torch = torch_cuda
    from synth import icosphere, planewave_batch
    from oracle import operator as op, excitation, solve as osolve
    from paper_2009_02281_gb300 import Context, Gnn, EFIE, F64, PRECOND_LEARNED, PRECOND_DIAG
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (16, 16, 16), order=2, formulation=EFIE)
    freq = 299792458.0 / 2
    net = Gnn(EFIE)
    net.init_params(0)
    losses = net.fit([(ctx, freq)], steps=1500, nprobe=16, lr=2e-3, clip=1.0, seed=1)
    assert np.mean(losses[-50:]) < 0.5 * losses[0]
    ctx.gnn_attach(net)
    dirs, pols = planewave_batch(2, seed=3)
    b = ctx.rhs_planewave(freq, dirs, pols)
    opts = dict(tol=1e-6, restart=300, max_iter=2000, inner_precision=F64)
    # the preconditioner's own iteration count (no trial against the diagonal one)
    xl, st_l, rc_l = ctx.solve(freq, b, precond=PRECOND_LEARNED, learned_trial=-1, **opts)
    xd, st_d, rc_d = ctx.solve(freq, b, precond=PRECOND_DIAG, **opts)
    assert rc_l == 0 and rc_d == 0
    # with the trial (default) the trained network wins it and finishes the solve
    _, st_t, rc_t = ctx.solve(freq, b, precond=PRECOND_LEARNED, **opts)
    assert rc_t == 0 and all(q["precond_used"] == PRECOND_LEARNED for q in st_t)
    it_l = [s["iterations"] for s in st_l]
    it_d = [s["iterations"] for s in st_d]
    print("loss", losses[0], np.mean(losses[-50:]), "iterations learned", it_l, "diag", it_d)
    assert sum(it_l) <= 0.85 * sum(it_d)
    prob = op.setup(xyz, tri, 2, (16, 16, 16), radius=3)
    A = op.dense_efie(prob, freq)
    for k in range(2):
        bo, _ = excitation.planewave_rhs(prob["rwg"], 2 * np.pi * freq / 299792458.0, dirs[k], pols[k])
        ref = osolve.lu_solve(A, bo)
        got = xl[k].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    net.close()
    ctx.close()


def test_untrained_network_loses_its_trial(torch_cuda):
    """A network with random parameters preconditions badly: the short trial against the
    diagonal preconditioner (judged by the true residual) hands the solve to the diagonal
    one, which reaches the dense-LU solution."""
    torch = torch_cuda
    from synth import icosphere, planewave_batch
    from oracle import operator as op, excitation, solve as osolve
    from paper_2009_02281_gb300 import Context, Gnn, EFIE, F64, PRECOND_LEARNED, PRECOND_DIAG
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (16, 16, 16), order=2, formulation=EFIE)
    freq = 299792458.0 / 2
    net = Gnn(EFIE)
    rng = np.random.default_rng(5)
    net.set_params((0.5 * rng.standard_normal(net.params().size)).astype(np.float32))
    ctx.gnn_attach(net)
    net.close()
    dirs, pols = planewave_batch(2, seed=3)
    b = ctx.rhs_planewave(freq, dirs, pols)
    opts = dict(tol=1e-6, restart=300, max_iter=2000, inner_precision=F64)
    _, st_n, _ = ctx.solve(freq, b, precond=PRECOND_LEARNED, learned_trial=-1, **opts)
    x, st, rc = ctx.solve(freq, b, precond=PRECOND_LEARNED, **opts)
    _, st_d, _ = ctx.solve(freq, b, precond=PRECOND_DIAG, **opts)
    assert rc == 0
    assert all(q["precond_used"] == PRECOND_DIAG for q in st)
    it = sum(q["iterations"] for q in st)
    # the trial costs two short cycles at most on top of the diagonal solve, and beats the bad network
    assert it <= sum(q["iterations"] for q in st_d) + 2 * 2 * 10
    assert it < sum(q["iterations"] for q in st_n)
    prob = op.setup(xyz, tri, 2, (16, 16, 16), radius=3)
    A = op.dense_efie(prob, freq)
    for k in range(2):
        bo, _ = excitation.planewave_rhs(prob["rwg"], 2 * np.pi * freq / 299792458.0, dirs[k], pols[k])
        ref = osolve.lu_solve(A, bo)
        assert np.linalg.norm(x[k].cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)
    ctx.close()
