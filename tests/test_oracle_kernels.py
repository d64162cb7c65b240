"""Pins for the closed-form triangle potentials and the Green's function kernels.

Independent references: brute-force (subdivided) Gauss quadrature, polar
integration for in-plane points, central finite differences, the Taylor limit
of Eq. hgfdtaylor, and symbolic derivatives from sympy for Eqs. Dhgf / Dghgf.
"""

import math

import numpy as np
import pytest

from oracle import potentials as pot, greens, quadrature as qd


TRI = (np.array([0.1, -0.2, 0.05]), np.array([1.2, 0.1, -0.1]), np.array([0.3, 0.9, 0.2]))


def _subdivide(v0, v1, v2, level):
    tris = [(v0, v1, v2)]
    for _ in range(level):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = nxt
    return tris


def _brute(r, v0, v1, v2, level=3, q=12):
    bary, w = qd.triangle_rule(q)
    I1 = 0.0
    J = np.zeros(3)
    G = np.zeros(3)
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm)
    rho = r - np.dot(r - v0, nrm) * nrm
    for a, b, c in _subdivide(v0, v1, v2, level):
        A = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        pts = bary @ np.stack([a, b, c])
        R = np.linalg.norm(r - pts, axis=1)
        I1 += A * np.sum(w / R)
        J += A * np.einsum("q,qk->k", w / R, pts - rho)
        G += -A * np.einsum("q,qk->k", w / R ** 3, r - pts)
    return I1, J, G


@pytest.mark.parametrize("r", [np.array([0.4, 0.3, 2.0]), np.array([-1.5, 0.2, 0.3]),
                               np.array([0.5, 0.3, -0.7]), np.array([2.0, 2.0, 0.0])])
def test_potentials_vs_quadrature(r):
    I1, J, G, _ = pot.tri_potentials(r, *TRI)
    bI, bJ, bG = _brute(r, *TRI)
    assert I1 == pytest.approx(bI, rel=1e-9)
    assert np.allclose(J, bJ, rtol=0, atol=1e-9 * np.abs(bJ).max())
    assert np.allclose(G, bG, rtol=0, atol=1e-8 * np.abs(bG).max())


def test_gradient_vs_finite_difference():
    r = np.array([0.45, 0.25, 0.12])       # close above the triangle
    _, _, G, _ = pot.tri_potentials(r, *TRI)
    h = 1e-6
    fd = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd[a] = (pot.tri_potentials(r + e, *TRI)[0] - pot.tri_potentials(r - e, *TRI)[0]) / (2 * h)
    assert np.allclose(G, fd, rtol=0, atol=1e-6 * np.abs(G).max())


def test_in_plane_point_polar_integration():
    """For a point inside T (d = 0): I1 = sum over edges of int rho_edge(theta) dtheta."""
    v0, v1, v2 = TRI
    r = (v0 + 2 * v1 + 1.5 * v2) / 4.5
    I1, J, G, _ = pot.tri_potentials(r, v0, v1, v2)
    x, w = np.polynomial.legendre.leggauss(60)
    s_ = 0.5 * (x + 1)
    tot = 0.0
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        # sub-triangle (r, a, b) in polar form: int rho(theta) dtheta, with the angle
        # parametrised by the edge point P(s) = a + s (b - a): dtheta = |(P-r) x (b-a)| / |P-r|^2 ds
        P = a[None, :] + s_[:, None] * (b - a)[None, :]
        d = P - r
        tot += 0.5 * np.sum(w * np.linalg.norm(np.cross(d, b - a), axis=1) / np.linalg.norm(d, axis=1))
    assert I1 == pytest.approx(tot, rel=1e-10)
    # the principal-value normal component vanishes in the plane
    nrm = np.cross(v1 - v0, v2 - v0)
    assert abs(np.dot(G, nrm)) < 1e-12


def test_solid_angle_limit():
    """Just above the interior the normal derivative of I1 tends to -2 pi (solid angle 2 pi)."""
    v0, v1, v2 = TRI
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm)
    c = (v0 + v1 + v2) / 3
    _, _, G, _ = pot.tri_potentials(c + 1e-9 * nrm, v0, v1, v2)
    assert np.dot(G, nrm) == pytest.approx(-2 * np.pi, rel=1e-6)


def test_green_split_and_self_term():
    k = 2.3
    r = np.array([1e-3, 0.1, 1.0, 4.0])
    assert np.allclose(greens.G(k, r), greens.G_s(r) + greens.G_d(k, r), rtol=1e-14)
    # Eq. Hdmm: G_d -> -jk / (4 pi) as r -> 0
    assert greens.G_d(k, 1e-9) == pytest.approx(-1j * k / (4 * np.pi), rel=1e-7)
    H = greens.kernel_table(k, np.array([4, 5, 3]), np.array([0.1, 0.2, 0.3]))
    assert H[2, 4, 3] == -1j * k / (4 * np.pi)
    # sample at offset (1, 0, 0): r = 0.1
    assert H[2, 4, 4] == pytest.approx(np.exp(-1j * k * 0.1) / (4 * np.pi * 0.1), rel=1e-14)


def test_grad_kernel_vs_finite_difference():
    k = 1.7
    n = np.array([3, 3, 3])
    h = np.array([0.3, 0.25, 0.4])
    Hg = greens.grad_kernel_table(k, n, h)
    d = np.array([1, -2, 1])
    rv = d * h
    e = 1e-6
    for a in range(3):
        ea = np.zeros(3)
        ea[a] = e
        fd = (greens.G(k, np.linalg.norm(rv + ea)) - greens.G(k, np.linalg.norm(rv - ea))) / (2 * e)
        assert Hg[a][d[2] + 2, d[1] + 2, d[0] + 2] == pytest.approx(fd, rel=1e-7)
    assert np.all(Hg[:, 2, 2, 2] == 0)
    # Eq. gH00: |grad G_d| -> k^2 / (8 pi) as r -> 0
    t = 1e-5
    assert abs(greens.gradgd_radial(t)) == pytest.approx(1 / (8 * np.pi), rel=1e-4)


def test_derivative_formulas_vs_sympy():
    sympy = pytest.importorskip("sympy")
    th = sympy.symbols("theta", positive=True)
    gd = (sympy.exp(-sympy.I * th) - 1) / (4 * sympy.pi * th)
    F = ((1 + sympy.I * th) * sympy.exp(-sympy.I * th) - 1) / (4 * sympy.pi * th ** 2)
    for n in (1, 2, 3):
        d1 = sympy.diff(gd, th, n + 1)
        d2 = sympy.diff(F, th, n + 1)
        for t in (0.3, 1.1, 3.7):
            ref1 = complex(d1.subs(th, t).evalf())
            ref2 = complex(d2.subs(th, t).evalf())
            assert greens.dn_Gd(n, t) == pytest.approx(ref1, rel=1e-10)
            assert greens.dn_gradGd(n, t) == pytest.approx(ref2, rel=1e-10)


@pytest.mark.parametrize("spl", [10, 20, 30])
def test_interpolation_error_within_bound(spl):
    """Sec. IV-A / Figs. 2-3: order-2 Lagrange interpolation of G_d and grad G_d stays under B_n."""
    n = 2
    dth = 2 * np.pi / spl
    for func, dfunc in ((greens.gd_radial, greens.dn_Gd), (greens.gradgd_radial, greens.dn_gradGd)):
        for start in (0.05, 0.5, 1.5):
            nodes = start + dth * np.arange(n + 1)
            xs = np.linspace(nodes[0], nodes[-1], 101)
            err = greens.lagrange_interp_error(func, nodes, xs).max()
            bound = greens.interp_bound(dfunc, n, nodes[0], nodes[-1])
            assert err <= bound * (1 + 1e-9)
    # refinement lowers the error (controllable via grid refinement)
