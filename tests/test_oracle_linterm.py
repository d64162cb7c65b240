"""Pins of the linear-term modification oracle (Sec. III-A-3, Eqs. linterm and Lmatdecomplin).

* the closed-form inner integrals of |r - r'| against subdivided product quadrature,
* the mean distance of two random points in an equilateral triangle, (4 + 3 ln 3) / 20,
* the precorrection against the k^2 Taylor coefficient of the grid's own kernel table,
* the direct integrals against the k^2 Taylor coefficient of the dense MoM matrix,
* the paper's claim: the modification brings overlapping entries closer to direct integration.
"""

import numpy as np
import pytest

from oracle import linterm, mom
from oracle import operator as op
from oracle.quadrature import triangle_rule, map_points
from oracle.rwg import rwg_arrays
from synth import icosphere

C0 = 299792458.0


def _subdivide(v, levels):
    tris = [v]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(t) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]
        tris = nxt
    return tris


def _brute_r_potentials(r, v, levels=4, q=10):
    bary, w = triangle_rule(q)
    I = 0.0
    M = np.zeros(3)
    for t in _subdivide(v, levels):
        area = 0.5 * np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0]))
        p = map_points(bary, t[0], t[1], t[2])
        R = np.linalg.norm(p - r, axis=1)
        I += area * np.sum(w * R)
        M += area * np.sum((w * R)[:, None] * p, axis=0)
    return I, M


@pytest.mark.parametrize("where", ["above", "outside", "far", "in_plane", "near_vertex"])
def test_r_potentials_vs_subdivided_quadrature(where):
    v = np.array([[0.1, 0.2, 0.3], [1.2, -0.1, 0.5], [0.4, 0.9, -0.2]])
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    c = v.mean(0)
    r = {"above": c + 0.3 * n, "outside": c + 0.9 * (v[1] - v[2]) + 0.05 * n, "far": np.array([2.0, 1.0, 1.0]),
         "in_plane": 0.5 * v[0] + 0.3 * v[1] + 0.2 * v[2], "near_vertex": 0.999 * v[0] + 0.001 * v[1]}[where]
    IR, JR, rho = linterm.r_potentials(r, v[0], v[1], v[2])
    Ib, Mb = _brute_r_potentials(r, v)
    Jb = Mb - rho * Ib
    assert abs(IR - Ib) <= 1e-7 * Ib
    assert np.abs(JR - Jb).max() <= 1e-7 * np.abs(Jb).max()


def test_mean_distance_in_equilateral_triangle():
    """E|X - Y| for X, Y uniform on a unit equilateral triangle is (4 + 3 ln 3) / 20."""
    v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, np.sqrt(3.0) / 2.0, 0.0]])
    area = np.sqrt(3.0) / 4.0
    bary, w = triangle_rule(linterm.Q_LIN)
    p = map_points(bary, v[0], v[1], v[2])
    IR, _, _ = linterm.r_potentials(p, v[0], v[1], v[2])
    mean = np.sum(w * IR) / area
    assert abs(mean - (4.0 + 3.0 * np.log(3.0)) / 20.0) <= 1e-5 * mean


@pytest.fixture(scope="module")
def sphere():
    xyz, tri = icosphere(1)
    prob = op.setup(xyz, tri, 2, (8, 8, 8), radius=3)
    return prob, linterm.lin_matrices(prob)


def test_overlapping_pairs_are_the_shared_triangle_pairs(sphere):
    prob, (rows, cols, _, _) = sphere
    T, _, _, _ = rwg_arrays(prob["rwg"])
    N = prob["N"]
    want = {(m, n) for m in range(N) for n in range(N) if set(T[m].tolist()) & set(T[n].tolist())}
    got = set(zip(rows.tolist(), cols.tolist()))
    assert got == want
    assert all(np.diff(rows) >= 0)


def test_precorrection_is_k2_coefficient_of_grid_kernel(sphere):
    """Re H(k) = H_s + k^2 H_lin + O(k^4): the grid matrices' k^2 coefficient on the pairs is L_lin,P."""
    prob, (rows, cols, _, _) = sphere
    PA, PP = linterm.lin_precorrection(prob["lam"], prob["anc"], prob["grid"], rows, cols)
    k1, k2 = 0.02, 0.01
    A1, P1, _ = op._grid_matrices(prob, k1, False)
    A2, P2, _ = op._grid_matrices(prob, k2, False)
    cA = (A1.real - A2.real)[rows, cols] / (k1 ** 2 - k2 ** 2)
    cP = (P1.real - P2.real)[rows, cols] / (k1 ** 2 - k2 ** 2)
    assert np.abs(cA - PA).max() <= 1e-3 * np.abs(PA).max()
    assert np.abs(cP - PP).max() <= 1e-3 * np.abs(PP).max()


def test_direct_is_k2_coefficient_of_mom(sphere):
    """Re G(k) = G_s + k^2 G_lin + O(k^4): the MoM matrices' k^2 coefficient on the pairs is L_lin.

    The MoM integrates the non-smooth dynamic part with a plain product rule, so
    this holds to that rule's accuracy on the coincident triangles (about 1e-2).
    """
    prob, (rows, cols, _, _) = sphere
    LA, LP = linterm.lin_direct(prob["rwg"], rows, cols)
    f1, f2 = 0.02 * C0 / (2 * np.pi), 0.01 * C0 / (2 * np.pi)
    _, A1, P1 = mom.dense_efie_mom(prob["rwg"], f1)
    _, A2, P2 = mom.dense_efie_mom(prob["rwg"], f2)
    k1, k2 = 0.02, 0.01
    cA = (A1.real - A2.real)[rows, cols] / (k1 ** 2 - k2 ** 2)
    cP = (P1.real - P2.real)[rows, cols] / (k1 ** 2 - k2 ** 2)
    assert np.abs(cA - LA).max() <= 2e-2 * np.abs(LA).max()
    assert np.abs(cP - LP).max() <= 2e-2 * np.abs(LP).max()
    assert np.corrcoef(cA, LA)[0, 1] > 0.999 and np.corrcoef(cP, LP)[0, 1] > 0.999


def test_direct_symmetry(sphere):
    prob, (rows, cols, _, _) = sphere
    LA, LP = linterm.lin_direct(prob["rwg"], rows, cols)
    ta, tp = linterm.lin_direct(prob["rwg"], cols, rows)
    assert np.abs(LA - ta).max() <= 1e-5 * np.abs(LA).max()
    assert np.abs(LP - tp).max() <= 1e-5 * np.abs(LP).max()


def _product_rule_lin(rwg, rows, cols, q=5):
    """What a product Gauss rule on both triangles gives for the k^2 G_lin part (the dense MoM's treatment)."""
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri = rwg["xyz"], rwg["tri"]
    bary, w = triangle_rule(q)
    LA = np.zeros(len(rows))
    LP = np.zeros(len(rows))
    for i, (m, n) in enumerate(zip(rows, cols)):
        for a in range(2):
            rm = map_points(bary, *xyz[tri[T[m, a]]])
            fm = S[a] * C[m, a] * (rm - P[m, a])
            for b in range(2):
                rn = map_points(bary, *xyz[tri[T[n, b]]])
                fn = S[b] * C[n, b] * (rn - P[n, b])
                g = -np.linalg.norm(rm[:, None] - rn[None], axis=-1) / (8 * np.pi)
                ww = rwg["area"][T[m, a]] * rwg["area"][T[n, b]] * w[:, None] * w[None]
                LA[i] += np.sum(ww * g * (fm @ fn.T))
                LP[i] += S[a] * 2 * C[m, a] * S[b] * 2 * C[n, b] * np.sum(ww * g)
    return LA, LP


@pytest.mark.parametrize("frac,gain", [(0.125, 10.0), (0.25, 5.0)])
def test_modification_improves_overlapping_entries(sphere, frac, gain):
    """Overlapping entries against direct integration: the error drops by `gain` or more.

    The reference is the dense MoM with the k^2 G_lin part of its overlapping
    entries integrated with the closed-form inner integrals instead of the plain
    product rule (whose error on that non-smooth part is of the same order as
    the effect measured here).
    """
    prob, lin = sphere
    rows, cols = lin[0], lin[1]
    LAd, LPd = linterm.lin_direct(prob["rwg"], rows, cols)
    LAq, LPq = _product_rule_lin(prob["rwg"], rows, cols)
    f = frac * C0
    w, regs = op.materials(f, 1.0)
    mu, _, k = regs[0]
    Zr = mom.dense_efie_mom(prob["rwg"], f)[0]
    Zr[rows, cols] += 1j * w * mu * (k * k * (LAd - LAq) - (LPd - LPq))
    Z0 = op.dense_efie(prob, f)
    Z1 = linterm.dense_efie_lin(prob, f, lin=lin)
    ref = np.linalg.norm(Zr[rows, cols])
    e0 = np.linalg.norm((Z0 - Zr)[rows, cols]) / ref
    e1 = np.linalg.norm((Z1 - Zr)[rows, cols]) / ref
    assert e1 * gain <= e0
    assert np.linalg.norm(Z1 - Zr) < np.linalg.norm(Z0 - Zr)


def test_matvec_matches_dense(sphere):
    from synth import random_complex
    prob, lin = sphere
    f = 0.3 * C0
    x = random_complex((prob["N"],), seed=4)
    y = linterm.matvec_efie_lin(prob, f, x, lin=lin)
    Z = linterm.dense_efie_lin(prob, f, lin=lin)
    assert np.linalg.norm(y - Z @ x) <= 1e-12 * np.linalg.norm(y)


def test_pmchwt_with_equal_media_doubles_the_efie_term(sphere):
    """With identical media the two regions' L terms coincide: the E rows gain twice the EFIE term."""
    from synth import random_complex
    prob, lin = sphere
    N = prob["N"]
    f = 0.3 * C0
    xJ = random_complex((N,), seed=6)
    x = np.concatenate([xJ, np.zeros(N, dtype=np.complex128)])
    dP = linterm.matvec_pmchwt_lin(prob, f, x, 1.0, 1.0, lin=lin) - op.matvec_pmchwt(prob, f, x, 1.0, 1.0)
    dE = linterm.matvec_efie_lin(prob, f, xJ, lin=lin) - op.matvec_efie(prob, f, xJ)
    assert np.linalg.norm(dP[:N] - 2 * dE) <= 1e-12 * np.linalg.norm(dE)
    assert np.linalg.norm(dP[N:]) == 0.0
    xM = np.concatenate([np.zeros(N, dtype=np.complex128), xJ])
    dM = linterm.matvec_pmchwt_lin(prob, f, xM, 1.0, 1.0, lin=lin) - op.matvec_pmchwt(prob, f, xM, 1.0, 1.0)
    # eta0^2 j w eps0 = j w mu0: the H rows gain the same as the E rows
    assert np.linalg.norm(dM[N:] - 2 * dE) <= 1e-12 * np.linalg.norm(dE)
