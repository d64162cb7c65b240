"""Pins for the oracle's static near matrices, precorrection and assembled AIMx operator.

References other than the oracle code: brute-force product quadrature for
separated pairs, explicit loops for the precorrection, exact zeros of the
principal-value K on a flat face, symmetry/reciprocity of the Galerkin
operators, dense MoM by direct integration, and the Mie series.
"""

import numpy as np
import pytest

from synth import icosphere, box
from oracle import operator as op, static, grid as gm, greens, quadrature as qd, rwg as rw
from oracle import mom, mie, excitation, farfield, solve
from oracle.constants import C0, MU0, ETA0


def _brute_static(r, m, n, q=14):
    """Product Gauss quadrature of L^A_s, L^Phi_s and K_s for separated bases."""
    T, P, C, S = rw.rwg_arrays(r)
    xyz, tri, area = r["xyz"], r["tri"], r["area"]
    bary, w = qd.triangle_rule(q)
    LA = LP = KK = 0.0
    for so in range(2):
        to = T[m, so]
        ro = bary @ xyz[tri[to]]
        wo = w * area[to]
        fo = S[so] * C[m, so] * (ro - P[m, so])
        for ss in range(2):
            ts = T[n, ss]
            rs = bary @ xyz[tri[ts]]
            ws = w * area[ts]
            fs = S[ss] * C[n, ss] * (rs - P[n, ss])
            Rv = ro[:, None, :] - rs[None, :, :]
            R = np.linalg.norm(Rv, axis=-1)
            g = 1 / (4 * np.pi * R)
            LA += np.einsum("i,j,ij,ik,jk->", wo, ws, g, fo, fs)
            LP += S[so] * S[ss] * 4 * C[m, so] * C[n, ss] * np.einsum("i,j,ij->", wo, ws, g)
            gg = -Rv / (4 * np.pi * R[..., None] ** 3)
            KK += np.einsum("i,j,ik,ijk->", wo, ws, fo, np.cross(gg, fs[None, :, :]))
    return LA, LP, KK


def test_static_direct_vs_product_quadrature(small_sphere):
    r = small_sphere["rwg"]
    c = r["center"]
    pairs = [(0, int(np.argmax(np.linalg.norm(c - c[0], axis=1)))), (5, 60), (11, 97)]
    for m, n in pairs:
        if np.linalg.norm(c[m] - c[n]) < 0.6:
            continue
        LA, LP, KK = static.static_direct(r, np.array([m]), np.array([n]), q=12)
        bA, bP, bK = _brute_static(r, m, n)
        assert LA[0] == pytest.approx(bA, rel=1e-8)
        assert LP[0] == pytest.approx(bP, rel=1e-8)
        assert KK[0] == pytest.approx(bK, rel=1e-7, abs=1e-12)


def test_static_symmetry(small_sphere):
    """L^A_s, L^Phi_s and K_s are symmetric in (m, n) (Galerkin, W = P^T); quadrature-limited."""
    r = small_sphere["rwg"]
    rows = small_sphere["near"]["rows"]
    cols = small_sphere["cols"]
    LA, LP, KK = static.static_direct(r, rows, cols, q=12)
    LA2, LP2, KK2 = static.static_direct(r, cols, rows, q=12)
    assert np.abs(LA - LA2).max() < 1e-5 * np.abs(LA).max()
    assert np.abs(LP - LP2).max() < 5e-5 * np.abs(LP).max()
    # K's outer integrand is log-singular on shared edges/vertices, so the 12-point
    # rule converges slowly there; away from touching triangles symmetry is tight
    T = np.stack([r["tp"], r["tm"]], 1)
    tri = r["tri"]
    verts = [set(tri[T[i]].ravel()) for i in range(r["n"])]
    touch = np.array([len(verts[a] & verts[b]) > 0 for a, b in zip(rows, cols)])
    assert np.abs(KK - KK2)[~touch].max() < 1e-6 * np.abs(KK).max()
    assert np.abs(KK - KK2)[touch].max() < 5e-2 * np.abs(KK).max()


def test_k_static_zero_on_flat_face():
    """Principal value of K_s vanishes for RWG pairs lying in one plane (rhat x f normal to f)."""
    xyz, tri = box([0, 0, 0], [1, 1, 1], [3, 3, 3])
    r = rw.build_rwg(xyz, tri)
    T = np.stack([r["tp"], r["tm"]], 1)
    nz = np.abs(r["normal"][:, 2]) > 0.99
    on_top = [n for n in range(r["n"]) if all(nz[T[n]]) and
              all(abs(xyz[tri[T[n, s]], 2].mean() - 1) < 1e-12 for s in range(2))]
    m = np.array([a for a in on_top for b in on_top])
    n = np.array([b for a in on_top for b in on_top])
    _, _, KK = static.static_direct(r, m, n)
    assert np.abs(KK).max() < 1e-14


def test_precorrection_vs_loops(small_sphere):
    lam, anc, g = small_sphere["lam"], small_sphere["anc"], small_sphere["grid"]
    off = gm.stencil_offsets(2)
    rows = np.array([0, 3, 40])
    cols = np.array([0, 7, small_sphere["cols"][small_sphere["row_ptr"][40] + 2]])
    PA, PP, PK = static.precorrection(lam, anc, g, rows, cols, 3)
    h = g["h"]
    for i, (m, n) in enumerate(zip(rows, cols)):
        a = b = k = 0.0
        for u in range(27):
            for v in range(27):
                d = (anc[m] + off[u]) - (anc[n] + off[v])
                rv = d * h
                R = np.linalg.norm(rv)
                hs = 0.0 if R == 0 else 1 / (4 * np.pi * R)
                hg = np.zeros(3) if R == 0 else -rv / (4 * np.pi * R ** 3)
                a += hs * np.dot(lam[m, u, :3], lam[n, v, :3])
                b += hs * lam[m, u, 3] * lam[n, v, 3]
                k += np.dot(lam[m, u, :3], np.cross(hg, lam[n, v, :3]))
        assert PA[i] == pytest.approx(a, rel=1e-12)
        assert PP[i] == pytest.approx(b, rel=1e-12)
        assert PK[i] == pytest.approx(k, rel=1e-10, abs=1e-15)


def test_direct_sum_point_source():
    """out = H * delta reproduces the kernel samples (definition of the Toeplitz product)."""
    n = np.array([5, 4, 3])
    h = np.array([0.2, 0.3, 0.25])
    H = greens.kernel_table(1.3, n, h)
    g = np.zeros((1, 3, 4, 5), dtype=complex)
    g[0, 1, 2, 3] = 1.0
    out = op.conv_full(H, g)
    for z in range(3):
        for y in range(4):
            for x in range(5):
                assert out[0, z, y, x] == H[z - 1 + 2, y - 2 + 3, x - 3 + 4]
    nodes = np.array([[0, 0, 0], [4, 3, 2], [3, 2, 1]])
    gr = np.random.default_rng(3).standard_normal((2, 3, 4, 5)) + 0j
    full = op.conv_full(H, gr)
    part = op.conv_nodes(H, gr, nodes)
    for i, (x, y, z) in enumerate(nodes):
        assert np.allclose(part[:, i], full[:, z, y, x], rtol=1e-13)


def test_efie_reciprocity_and_matvec(small_sphere):
    f = 2.0 * C0 / (2 * np.pi)      # k = 2 rad/m
    Z = op.dense_efie(small_sphere, f)
    assert np.abs(Z - Z.T).max() < 1e-3 * np.abs(Z).max()   # quadrature-limited near symmetry
    x = np.random.default_rng(0).standard_normal(small_sphere["N"]) + 0j
    assert np.allclose(op.matvec_efie(small_sphere, f, x), Z @ x, rtol=1e-12, atol=1e-12 * np.abs(Z @ x).max())


def test_pmchwt_reciprocity_and_sampled_rows(small_sphere):
    f = 1.0 * C0 / (2 * np.pi)
    Z = op.dense_pmchwt(small_sphere, f, 1.0, 4.0)
    N = small_sphere["N"]
    D = np.r_[np.ones(N), -np.ones(N)]
    DZ = D[:, None] * Z
    assert np.abs(DZ - DZ.T).max() < 3e-3 * np.abs(Z).max()
    x = np.random.default_rng(1).standard_normal(2 * N) + 1j * np.random.default_rng(2).standard_normal(2 * N)
    y = Z @ x
    assert np.allclose(op.matvec_pmchwt(small_sphere, f, x, 1.0, 4.0), y, rtol=1e-12, atol=1e-12 * np.abs(y).max())
    xyz, tri = icosphere(1)
    rows = np.array([2, 50, 119])
    ps = op.setup(xyz, tri, 2, [8, 8, 8], radius=3, near_rows=rows)
    ys = op.matvec_pmchwt(ps, f, x, 1.0, 4.0, rows=rows)
    assert np.allclose(ys, np.r_[y[rows], y[N + rows]], rtol=1e-12, atol=1e-12 * np.abs(y).max())


@pytest.fixture(scope="module")
def mom_l2(sphere_l2):
    """Dense MoM of the level-2 sphere at mean edge length 0.1 lambda."""
    r = sphere_l2["rwg"]
    f = C0 / (10 * r["length"].mean())
    Zm, _, _ = mom.dense_efie_mom(r, f)
    return f, Zm


def test_aimx_converges_to_mom_with_order(mom_l2):
    """AIMx error against dense MoM falls as the stencil order rises (Sec. IV, E2 trend)."""
    xyz, tri = icosphere(2)
    f, Zm = mom_l2
    errs = []
    for order, nn in ((1, 10), (2, 10), (3, 12), (2, 16)):
        p = op.setup(xyz, tri, order, [nn] * 3, radius=2)
        Z = op.dense_efie(p, f)
        errs.append(np.linalg.norm(Z - Zm) / np.linalg.norm(Zm))
    assert errs[0] > errs[1] > errs[2]
    assert errs[3] < errs[1]            # grid refinement at fixed order
    assert errs[1] < 2e-2


def test_diagonal_error_below_one_percent(sphere_l2, mom_l2):
    """Overlapping basis/test error stays below 1% at edge length ~0.1 lambda (Sec. IV-B)."""
    f, Zm = mom_l2
    Z = op.dense_efie(sphere_l2, f)
    d = np.abs(np.diag(Z) - np.diag(Zm)) / np.abs(np.diag(Zm))
    assert d.max() < 1e-2


def test_pec_sphere_rcs_vs_mie(sphere_l2):
    k = 1.0
    f = k * C0 / (2 * np.pi)
    Z = op.dense_efie(sphere_l2, f)
    VE, _ = excitation.planewave_rhs(sphere_l2["rwg"], k, [0, 0, 1], [1, 0, 0])
    J = solve.lu_solve(Z, VE)
    th = np.linspace(0.2, np.pi - 0.2, 9)
    for phi in (0.0, np.pi / 2):
        dirs = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], 1)
        E = farfield.far_field(sphere_l2["rwg"], J, k, 2 * np.pi * f, MU0, dirs)
        s = farfield.rcs(E)
        ref = mie.bistatic_rcs(k, 1.0, th, phi)
        assert np.max(np.abs(s - ref) / ref.max()) < 0.06


def test_dielectric_sphere_rcs_vs_mie(sphere_l2):
    """PMCHWT signs are pinned by the dielectric Mie series."""
    k0 = 0.6
    f = k0 * C0 / (2 * np.pi)
    Z = op.dense_pmchwt(sphere_l2, f, 1.0, 4.0)
    VE, VH = excitation.planewave_rhs(sphere_l2["rwg"], k0, [0, 0, 1], [1, 0, 0], eta=ETA0)
    x = solve.lu_solve(Z, np.r_[VE, ETA0 * VH])
    N = sphere_l2["N"]
    th = np.linspace(0.2, np.pi - 0.2, 9)
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    E = farfield.far_field(sphere_l2["rwg"], x[:N], k0, 2 * np.pi * f, MU0, dirs, M=ETA0 * x[N:])
    s = farfield.rcs(E)
    ref = mie.bistatic_rcs(k0, 1.0, th, 0.0, eps_r=4.0)
    assert np.max(np.abs(s - ref) / ref.max()) < 0.08


def test_mie_pec_small_sphere_rayleigh():
    """Rayleigh limit of the PEC backscatter: sigma / (pi a^2) -> 9 (ka)^4."""
    ka = 0.01
    s = mie.bistatic_rcs(ka, 1.0, np.array([np.pi]), 0.0)[0]
    assert s / np.pi == pytest.approx(9 * ka ** 4, rel=1e-3)


def test_gmres_matches_lu(small_sphere):
    f = 2.0 * C0 / (2 * np.pi)
    Z = op.dense_efie(small_sphere, f)
    b = np.random.default_rng(5).standard_normal(small_sphere["N"]) + 0j
    x, it, rr = solve.gmres(lambda v: Z @ v, b, tol=1e-10, restart=50)
    assert rr <= 1e-10
    assert np.linalg.norm(x - solve.lu_solve(Z, b)) / np.linalg.norm(x) < 1e-8


def test_loop_currents_scalar_potential(small_sphere):
    """Divergence-free (loop) currents: the MoM scalar potential vanishes on them exactly; the
    AIMx one does not.

    A combination x of RWG functions with D x = 0 (D the RWG-to-triangle incidence, the discrete
    divergence) carries no charge, so L^Phi x = int int div f_m div'(sum x_n f_n) G = 0 for any
    kernel.  On a closed genus-0 surface the loop space has dimension N - T + 1 (Euler).  AIMx
    projects each basis onto its own stencil (moment matching, Sec. II-B), so the projected charges
    of neighbouring bases no longer cancel node by node: the grid charge P_rho x of a loop is not
    zero, only its moments up to the stencil order vanish.  The remainder acts as a high-order
    multipole source that the near correction removes only inside the near region, and the
    residue left in L^Phi x, amplified by 1/k^2 at small k h, swamps the vector-potential term of
    electrically small conductors (the case the AEFIE's charge form L^Phi = D^T P D avoids)."""
    import scipy.linalg as sl
    prob = small_sphere
    r = prob["rwg"]
    N, nt = r["n"], len(r["tri"])
    T, P, C, S = rw.rwg_arrays(r)
    D = np.zeros((nt, N))
    for n in range(N):
        D[T[n, 0], n] += r["length"][n]
        D[T[n, 1], n] -= r["length"][n]
    Q = sl.null_space(D)
    assert Q.shape[1] == N - nt + 1
    x = Q @ np.random.default_rng(1).standard_normal(Q.shape[1])
    k = 0.5
    _, LA, LP = mom.dense_efie_mom(r, k * C0 / (2 * np.pi))
    nP, nx = np.linalg.norm(LP, 2), np.linalg.norm(x)
    assert np.linalg.norm(LP @ x) <= 1e-12 * nP * nx
    # the loop's grid charge is not zero, but its moments up to the stencil order vanish ...
    grid = prob["grid"]
    g = gm.project(prob["lam"], prob["anc"], grid, x, fields=(3,))[0]
    Nx, Ny, Nz = grid["n"]
    zz, yy, xx = np.meshgrid(*(np.arange(n) * grid["h"][a] + grid["origin"][a] for a, n in ((2, Nz), (1, Ny), (0, Nx))),
                             indexing="ij")
    assert np.abs(g).max() > 1e-3 * np.abs(x).max() * np.abs(D).max()
    scale = np.sum(np.abs(g))
    for ax in range(grid["order"] + 1):
        for ay in range(grid["order"] + 1):
            for az in range(grid["order"] + 1):
                mom_ = np.sum(g * xx ** ax * yy ** ay * zz ** az)
                assert abs(mom_) <= 1e-12 * scale * max(1.0, np.abs(xx).max()) ** (ax + ay + az)
    # ... and the AIMx scalar potential of the loop leaves a residue far above rounding
    GA, GP, _ = op._grid_matrices(prob, k, False)
    LPa = op.near_dense(prob, "NP") + GP
    leak = np.linalg.norm(LPa @ x) / (nP * nx)
    assert 1e-6 < leak < 1e-2
