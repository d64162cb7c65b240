"""Pins for the FP64 reference of the learned preconditioner network.

Gradients from explicit backpropagation are checked against central finite
differences of the loss, for the scalar (EFIE) and 2x2-block (two-region)
output forms; the preconditioner application against an explicit dense
matrix; the network's orientation equivariance (C_mn -> s_m s_n C_mn when the
signed bases flip and the invariant features do not); the two-hop bases
against their definition summed term by term; the features' translation and
scale invariance and pair symmetries; and D^{-1} against the low-frequency
diagonal of the assembled operator.
"""

import numpy as np
import pytest

from oracle import gnn


def _graph(N, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for m in range(N):
        nb = set([m] + list(rng.choice(N, size=4, replace=False)))
        for n in sorted(nb):
            rows.append(m)
            cols.append(n)
    rows, cols = np.array(rows), np.array(cols)
    # make the pattern symmetric like the near relation
    pairs = set(zip(rows, cols)) | set(zip(cols, rows))
    pairs = sorted(pairs)
    return np.array([p[0] for p in pairs]), np.array([p[1] for p in pairs])


def _random_params(rng, K, width, layers):
    params = gnn.init_params(5, width=width, layers=layers, K=K)
    for k in ("E", "f", "G", "g", "u", "Ua"):
        params[k] = 0.3 * rng.standard_normal(params[k].shape)
    return params


@pytest.mark.parametrize("K", [2, 8])
def test_gradients_match_finite_differences(K):
    rng = np.random.default_rng(3)
    N = 12
    rows, cols = _graph(N, 1)
    width, layers = 6, 2
    params = _random_params(rng, K, width, layers)
    x = rng.standard_normal((N, gnn.NIN))
    e = rng.standard_normal((len(rows), gnn.NED))
    basis = rng.standard_normal((len(rows), gnn.NB))
    nunk = N if K == 2 else 2 * N
    if K == 2:
        dinv = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    else:
        dinv = rng.standard_normal((N, 2, 2)) + 1j * rng.standard_normal((N, 2, 2))
    Y = rng.standard_normal((3, nunk)) + 1j * rng.standard_normal((3, nunk))
    Z = rng.standard_normal((3, nunk)) + 1j * rng.standard_normal((3, nunk))
    args = (x, e, basis, rows, cols, dinv, Y, Z, K, layers)
    L, grads = gnn.loss_and_grads(params, *args)
    h = 1e-6
    for name in params:
        flat = params[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = gnn.loss_and_grads(params, *args)
            flat[idx] = old - h
            Lm, _ = gnn.loss_and_grads(params, *args)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = grads[name].reshape(-1)[idx]
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, idx)


@pytest.mark.parametrize("K", [2, 8])
def test_orientation_equivariance(K):
    """Flipping basis orientations (signed bases s_m s_n b, invariant features fixed) gives s_m s_n C."""
    rng = np.random.default_rng(4)
    N = 15
    rows, cols = _graph(N, 6)
    params = _random_params(rng, K, 8, 3)
    x = rng.standard_normal((N, gnn.NIN))
    e = rng.standard_normal((len(rows), gnn.NED))
    basis = rng.standard_normal((len(rows), gnn.NB))
    s = rng.choice([-1.0, 1.0], size=N)
    o, g, _ = gnn.forward(params, x, e, basis, rows, cols, 3)
    o2, g2, _ = gnn.forward(params, x, e, basis * (s[rows] * s[cols])[:, None], rows, cols, 3)
    assert np.allclose(o2, o * (s[rows] * s[cols])[:, None], rtol=1e-12, atol=1e-12)
    assert np.array_equal(g2, g)


@pytest.mark.parametrize("K", [2, 8])
def test_apply_precond_dense(K):
    rng = np.random.default_rng(7)
    N = 9
    rows, cols = _graph(N, 2)
    nunk = N if K == 2 else 2 * N
    o = rng.standard_normal((len(rows), K)) * (rows != cols)[:, None]
    g = rng.standard_normal((N, K))
    oc, gc = gnn.to_complex_blocks(o, g, K)
    if K == 2:
        dinv = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        C = np.zeros((N, N), complex)
        C[rows, cols] += oc
        C[np.arange(N), np.arange(N)] += gc
        M = np.diag(dinv) @ (np.eye(N) + C)
    else:
        dinv = rng.standard_normal((N, 2, 2)) + 1j * rng.standard_normal((N, 2, 2))
        C = np.zeros((2 * N, 2 * N), complex)
        Dm = np.zeros((2 * N, 2 * N), complex)
        for k, (m, n) in enumerate(zip(rows, cols)):
            for a in range(2):
                for b in range(2):
                    C[a * N + m, b * N + n] += oc[k, a, b]
        for m in range(N):
            for a in range(2):
                for b in range(2):
                    C[a * N + m, b * N + m] += gc[m, a, b]
                    Dm[a * N + m, b * N + m] = dinv[m, a, b]
        M = Dm @ (np.eye(2 * N) + C)
    v = rng.standard_normal(nunk) + 1j * rng.standard_normal(nunk)
    assert np.allclose(gnn.apply_precond(dinv, oc, gc, rows, cols, v, K), M @ v, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ network inputs on a real mesh

@pytest.fixture(scope="module")
def sphere_prob():
    from synth import icosphere
    from oracle import operator as op
    xyz, tri = icosphere(1)
    return op.setup(xyz, tri, 2, (8, 8, 8)), xyz, tri


def test_features_invariant_under_translation_and_scale(sphere_prob):
    from oracle import operator as op
    prob, xyz, tri = sphere_prob
    f = 2.0e8
    x0, e0, b0, r0, c0 = gnn.features(prob, f)
    g = prob["grid"]
    s, t = 3.0, np.array([0.7, -1.1, 2.3])
    prob2 = op.setup(xyz * s + t, tri, 2, (8, 8, 8), h=np.asarray(g["h"]) * s,
                     origin=np.asarray(g["origin"]) * s + t)
    x1, e1, b1, r1, c1 = gnn.features(prob2, f / s)
    assert np.array_equal(r0, r1) and np.array_equal(c0, c1)
    assert np.allclose(x0, x1, atol=1e-9)
    assert np.allclose(e0, e1, atol=1e-7)
    assert np.allclose(b0, b1, atol=1e-7)


def test_two_hop_bases_match_definition(sphere_prob):
    prob, _, _ = sphere_prob
    x, e, basis, rows, cols = gnn.features(prob, 2.0e8)
    N = prob["N"]
    pos = {(int(m), int(n)): i for i, (m, n) in enumerate(zip(rows, cols))}
    nbr = [[] for _ in range(N)]
    for m, n in zip(rows, cols):
        nbr[int(m)].append(int(n))
    deg = np.array([max(len(v) - 1, 1) for v in nbr], dtype=float)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(rows), size=40, replace=False):
        m, n = int(rows[i]), int(cols[i])
        for c, name in enumerate(gnn.BASES[3:]):
            a, b = "APK".index(name[0]), "APK".index(name[1])
            acc = 0.0
            for j in nbr[m]:
                if (j, n) in pos:
                    acc += basis[pos[(m, j)], a] * basis[pos[(j, n)], b]
            assert basis[i, 3 + c] == pytest.approx(acc / np.sqrt(deg[m] * deg[n]), rel=1e-12, abs=1e-15)


def test_edge_features_symmetry(sphere_prob):
    prob, _, _ = sphere_prob
    x, e, basis, rows, cols = gnn.features(prob, 2.0e8)
    pos = {(int(m), int(n)): i for i, (m, n) in enumerate(zip(rows, cols))}
    tr = np.array([pos[(int(n), int(m))] for m, n in zip(rows, cols)])
    assert np.allclose(e[tr, 0:3], -e[:, 0:3])
    # distance and k h are exactly symmetric; the static near values only to quadrature accuracy
    assert np.array_equal(e[tr, 3], e[:, 3]) and np.array_equal(e[tr, 15], e[:, 15])
    assert np.allclose(basis[tr, 0:2], basis[:, 0:2], atol=1e-3)
    assert np.allclose(basis[tr, 2], basis[:, 2], atol=2e-2)
    diag = rows == cols
    assert np.allclose(basis[diag, 0:2], 1.0)
    assert np.all(np.abs(x[:, 3:6]) <= 0.5 + 1e-12)
    assert np.all(e[:, [4, 5, 7, 8, 9, 10, 11, 12]] >= 0)


def test_diag_inverse_matches_low_frequency_operator_diagonal(sphere_prob):
    """At k h << 1 the AIMx self terms reduce to the static self terms (Eq. LAIMx)."""
    from oracle import operator as op
    prob, _, _ = sphere_prob
    f = 3.0e6
    d = 1.0 / gnn.diag_inverse(prob, f)
    Z = op.dense_efie(prob, f)
    assert np.allclose(d, np.diag(Z), rtol=2e-2)
    N = prob["N"]
    blk = np.linalg.inv(gnn.diag_inverse(prob, f, 1.0, 4.0))
    Zp = op.dense_pmchwt(prob, f, 1.0, 4.0)
    ref = np.stack([np.stack([np.diag(Zp[:N, :N]), np.diag(Zp[:N, N:])], -1),
                    np.stack([np.diag(Zp[N:, :N]), np.diag(Zp[N:, N:])], -1)], -2)
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    assert np.allclose(blk / scale, ref / scale, atol=2e-2)
