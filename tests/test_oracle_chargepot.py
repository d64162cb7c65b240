"""Pins for the charge-form scalar potential of the oracle (EFIE and two-region PMCHWT).

References other than the module itself: the Euler count of the loop space, the exact identity
L^Phi_s = D^T Pt_s D against the RWG static integrals, moments of the pulse weights against a
higher-order quadrature, the precorrection against explicit loops, the dense MoM scalar
potential, and the vanishing potential of divergence-free currents.
"""

import numpy as np
import pytest

from oracle import chargepot as cp, grid as gm, greens, mom, operator as op, static
from oracle.quadrature import triangle_rule, map_points
from oracle.constants import C0


@pytest.fixture(scope="module")
def ch1(small_sphere):
    return cp.setup_charge(small_sphere)


def test_incidence(small_sphere, ch1):
    r = small_sphere["rwg"]
    D = ch1["D"]
    nt, N = D.shape
    assert np.allclose(D.sum(axis=0), 0.0)                          # +l on T+, -l on T-
    assert np.allclose(np.abs(D).sum(axis=0), 2 * r["length"])
    assert np.linalg.matrix_rank(D) == nt - 1                        # closed surface: total charge 0
    assert N - np.linalg.matrix_rank(D) == N - nt + 1                # Euler: loop space dimension


def test_static_identity_against_rwg_integrals(small_sphere):
    """L^Phi_s(m, n) = sum_ij D_im Pt_s(i, j) D_jn on every pair, including the singular ones."""
    r = small_sphere["rwg"]
    N, nt = r["n"], len(r["tri"])
    ii, jj = np.meshgrid(np.arange(nt), np.arange(nt), indexing="ij")
    Ps = cp.static_pulse(r, ii.ravel(), jj.ravel()).reshape(nt, nt)
    mm, nn = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    LPs = static.static_direct(r, mm.ravel(), nn.ravel())[1].reshape(N, N)
    D = cp.incidence(r)
    assert np.abs(D.T @ Ps @ D - LPs).max() <= 1e-12 * np.abs(LPs).max()
    assert np.allclose(Ps, Ps.T, rtol=1e-2, atol=0)                  # symmetric up to the outer rule


def test_pulse_weight_moments(small_sphere, ch1):
    """sum_u Lp[u, t] (r_u - c)^alpha = A_t^-1 int_T (r - c)^alpha dS for alpha_i <= n."""
    r, g = small_sphere["rwg"], small_sphere["grid"]
    o = g["order"]
    off = gm.stencil_offsets(o)
    bary, w = triangle_rule(10)
    xyz, tri = r["xyz"], r["tri"]
    for t in (0, 17, 55):
        c = xyz[tri[t]].mean(axis=0)
        nodes = g["origin"] + (ch1["anc_t"][t] + off) * g["h"]
        q = map_points(bary, xyz[tri[t, 0]][None], xyz[tri[t, 1]][None], xyz[tri[t, 2]][None])[0]
        for a in range(o + 1):
            for b in range(o + 1):
                for e in range(o + 1):
                    lhs = np.sum(ch1["Lp"][t] * (nodes[:, 0] - c[0]) ** a * (nodes[:, 1] - c[1]) ** b
                                 * (nodes[:, 2] - c[2]) ** e)
                    rhs = np.sum(w * (q[:, 0] - c[0]) ** a * (q[:, 1] - c[1]) ** b * (q[:, 2] - c[2]) ** e)
                    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


def test_precorrection_vs_loops(small_sphere, ch1):
    g = small_sphere["grid"]
    off = gm.stencil_offsets(g["order"])
    Lp, anc = ch1["Lp"], ch1["anc_t"]
    span = ch1["radius"] + g["order"]
    Hs, _ = greens.static_offset_kernels(g["h"], span)
    picks = [0, 5, len(ch1["rows"]) // 2, len(ch1["rows"]) - 1]
    rows, cols = ch1["rows"][picks], ch1["cols"][picks]
    got = cp.pulse_precorrection(Lp, anc, g, rows, cols, ch1["radius"])
    for p, (i, j) in enumerate(zip(rows, cols)):
        want = 0.0
        for u in range(len(off)):
            for v in range(len(off)):
                d = anc[i] + off[u] - anc[j] - off[v] + span
                want += Lp[i, u] * Hs[d[2], d[1], d[0]] * Lp[j, v]
        assert abs(got[p] - want) <= 1e-13 * max(1e-30, abs(want))


def test_charge_form_against_mom_and_on_loops(small_sphere, ch1):
    """The AIMx charge form approximates the MoM scalar potential as well as the RWG form does, and
    gives divergence-free currents exactly zero potential where the RWG form leaves a residue."""
    import scipy.linalg as sl
    prob = small_sphere
    r = prob["rwg"]
    k = 0.5
    LPc = cp.lphi_charge_dense(prob, ch1, k)
    _, LA, LPm = mom.dense_efie_mom(r, k * C0 / (2 * np.pi))
    GA, GP, _ = op._grid_matrices(prob, k, False)
    LPr = op.near_dense(prob, "NP") + GP
    ec = np.linalg.norm(LPc - LPm) / np.linalg.norm(LPm)
    er = np.linalg.norm(LPr - LPm) / np.linalg.norm(LPm)
    assert ec < 5e-3 and ec < 3 * er
    x = sl.null_space(ch1["D"]) @ np.random.default_rng(1).standard_normal(r["n"] - len(r["tri"]) + 1)
    nP, nx = np.linalg.norm(LPm, 2), np.linalg.norm(x)
    assert np.linalg.norm(LPc @ x) <= 1e-12 * nP * nx
    assert np.linalg.norm(LPr @ x) > 1e-6 * nP * nx


def test_dense_efie_charge_solves_like_the_rwg_form_on_a_sphere(small_sphere, ch1):
    """Plane-wave currents on a sphere at k a = 0.5 against MoM: the charge form is the more
    accurate AIMx form (1.1e-3 against 2.5e-2 for the RWG form on this 8^3 grid), consistent with
    the 1/k^2 amplifying the RWG form's scalar-potential residue on the current's loop part."""
    from oracle.excitation import planewave_rhs
    prob = small_sphere
    r = prob["rwg"]
    f = 0.5 * C0 / (2 * np.pi)
    b = planewave_rhs(r, 0.5, [0, 0, 1.0], [1.0, 0, 0])
    b = b[0] if isinstance(b, tuple) else b
    Jm = np.linalg.solve(mom.dense_efie_mom(r, f)[0], b)
    Jc = np.linalg.solve(cp.dense_efie_charge(prob, ch1, f), b)
    Jr = np.linalg.solve(op.dense_efie(prob, f), b)
    ec = np.linalg.norm(Jc - Jm) / np.linalg.norm(Jm)
    er = np.linalg.norm(Jr - Jm) / np.linalg.norm(Jm)
    assert ec < 5e-3 and ec < 0.2 * er


def test_matvec_equals_dense(small_sphere, ch1):
    prob = small_sphere
    f = 0.5 * C0 / (2 * np.pi)
    x = np.random.default_rng(3).standard_normal(prob["N"]) + 1j * np.random.default_rng(4).standard_normal(prob["N"])
    y = cp.matvec_efie_charge(prob, ch1, f, x)
    Z = cp.dense_efie_charge(prob, ch1, f)
    assert np.linalg.norm(y - Z @ x) <= 1e-12 * np.linalg.norm(Z @ x)
    # and it differs from the RWG form only by the scalar-potential approximation
    yr = op.matvec_efie(prob, f, x)
    assert np.linalg.norm(y - yr) < 0.05 * np.linalg.norm(yr)


def test_sampled_rows_equal_full_product(small_sphere, ch1):
    prob = small_sphere
    f = 0.7 * C0 / (2 * np.pi)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(prob["N"]) + 1j * rng.standard_normal(prob["N"])
    rows = np.array([0, 7, 33, 64, prob["N"] - 1])
    y = cp.matvec_efie_charge(prob, ch1, f, x)
    ys = cp.matvec_efie_charge(prob, ch1, f, x, rows=rows)
    assert np.linalg.norm(ys - y[rows]) <= 1e-12 * np.linalg.norm(y[rows])


def test_pmchwt_charge_against_its_parts(small_sphere, ch1):
    """The two-region charge form assembled from pinned pieces: with M = 0 its electric rows are
    the sum over the regions of the charge-form EFIE products in each region's material, and its
    magnetic rows the RWG-form PMCHWT's (the K terms carry no scalar potential); with J = 0 its
    magnetic rows are sum_r eps_r x (charge-form EFIE of region r) (eta0^2 eps / mu = eps_r for
    mu = mu0) and its electric rows the RWG form's.  The dense matrix equals the product, and
    sampled rows equal the full product."""
    prob = small_sphere
    N = prob["N"]
    f = 0.6 * C0 / (2 * np.pi)
    eo, ei = 1.0, 4.0
    rng = np.random.default_rng(12)
    xJ = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xM = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    z = np.zeros(N, dtype=np.complex128)
    yJ = cp.matvec_pmchwt_charge(prob, ch1, f, np.r_[xJ, z], eo, ei)
    yM = cp.matvec_pmchwt_charge(prob, ch1, f, np.r_[z, xM], eo, ei)
    eJ = sum(cp.matvec_efie_charge(prob, ch1, f, xJ, eps_bg=e) for e in (eo, ei))
    eM = sum(e * cp.matvec_efie_charge(prob, ch1, f, xM, eps_bg=e) for e in (eo, ei))
    rJ = op.matvec_pmchwt(prob, f, np.r_[xJ, z], eo, ei)
    rM = op.matvec_pmchwt(prob, f, np.r_[z, xM], eo, ei)
    assert np.linalg.norm(yJ[:N] - eJ) <= 1e-12 * np.linalg.norm(eJ)
    assert np.linalg.norm(yJ[N:] - rJ[N:]) <= 1e-12 * np.linalg.norm(rJ[N:])
    assert np.linalg.norm(yM[N:] - eM) <= 1e-12 * np.linalg.norm(eM)
    assert np.linalg.norm(yM[:N] - rM[:N]) <= 1e-12 * np.linalg.norm(rM[:N])
    x = np.r_[xJ, xM]
    y = cp.matvec_pmchwt_charge(prob, ch1, f, x, eo, ei)
    Z = cp.dense_pmchwt_charge(prob, ch1, f, eo, ei)
    assert np.linalg.norm(Z @ x - y) <= 1e-11 * np.linalg.norm(y)
    rows = np.array([0, 5, N // 2, N - 1])
    ys = cp.matvec_pmchwt_charge(prob, ch1, f, x, eo, ei, rows=rows)
    assert np.linalg.norm(ys - np.r_[y[rows], y[N + rows]]) <= 1e-12 * np.linalg.norm(ys)
