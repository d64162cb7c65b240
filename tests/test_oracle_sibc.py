"""Pins for the surface-impedance and delta-gap port reference (oracle/sibc.py).

Gram entries against the closed form for products of linear functions on a
triangle; Gram symmetry and positive definiteness; the skin depth and surface
resistance of copper against their textbook values; the port functional
against the total current of a uniform surface current (perimeter of the cut,
with edge normals built independently of the port code); Y-parameter
reciprocity of the SIBC system.
"""

import numpy as np
import pytest

from oracle import sibc


def _bar(n=(8, 2, 2), size=(40e-6, 10e-6, 5e-6)):
    from synth import box
    return box([0, 0, 0], list(size), list(n))


def test_gram_matches_linear_closed_form():
    from oracle.rwg import build_rwg, rwg_arrays
    xyz, tri = _bar()
    rwg = build_rwg(xyz, tri)
    T, P, C, S = rwg_arrays(rwg)
    rng = np.random.default_rng(0)
    N = rwg["n"]
    checked = 0
    for m in rng.choice(N, size=40, replace=False):
        for n in range(N):
            ref = 0.0
            share = False
            for a in range(2):
                for b in range(2):
                    t = T[m, a]
                    if t != T[n, b]:
                        continue
                    share = True
                    v = rwg["xyz"][rwg["tri"][t]]
                    A = rwg["area"][t]
                    um = v - P[m, a]
                    un = v - P[n, b]
                    # int_T (r - p).(r - q) dS = A/12 [sum_i u_i.w_i + (sum u_i).(sum w_i)]
                    lin = A / 12.0 * (np.sum(um * un) + um.sum(0) @ un.sum(0))
                    ref += S[a] * S[b] * C[m, a] * C[n, b] * lin
            if share:
                got = sibc.gram(rwg, np.array([m]), np.array([n]))[0]
                assert got == pytest.approx(ref, rel=1e-10, abs=1e-12 * rwg["area"].max())
                checked += 1
    assert checked > 40


def test_gram_symmetric_positive_definite():
    from oracle.rwg import build_rwg
    xyz, tri = _bar()
    G = sibc.gram_dense(build_rwg(xyz, tri))
    assert np.allclose(G, G.T, rtol=1e-12, atol=0)
    assert np.linalg.eigvalsh(G).min() > 0


def test_copper_skin_depth_and_surface_resistance():
    sigma = 5.8e7
    f = 1e9
    w = 2 * np.pi * f
    delta = np.sqrt(2.0 / (w * 4e-7 * np.pi * sigma))
    assert delta == pytest.approx(2.09e-6, rel=2e-3)       # textbook copper skin depth at 1 GHz
    zs = sibc.surface_impedance(f, sigma)
    assert zs.real == pytest.approx(8.25e-3, rel=2e-3)     # R_s = sqrt(w mu / (2 sigma))
    assert zs.imag == pytest.approx(zs.real, rel=1e-12)


def test_port_current_of_uniform_surface_current():
    """A uniform current J0 x-hat on the bar's side faces crosses the gap plane x = L/2
    with total current J0 times the cut perimeter."""
    from oracle.rwg import build_rwg
    size = (40e-6, 10e-6, 5e-6)
    xyz, tri = _bar(size=size)
    rwg = build_rwg(xyz, tri)
    port = ([size[0] / 2, 0, 0], [1, 0, 0], [-1, -1, -1], [1, 1, 1])
    c = sibc.port_vector(rwg, port)
    ids = np.nonzero(c)[0]
    assert len(ids) > 0
    J0 = 2.5
    # RWG coefficient = normal component of J across the edge, from T+ to T-,
    # with the in-plane edge normal built from T+'s face normal
    x = np.zeros(rwg["n"])
    for m in ids:
        a, b = rwg["xyz"][rwg["ea"][m]], rwg["xyz"][rwg["eb"][m]]
        t = (b - a) / np.linalg.norm(b - a)
        nf = rwg["normal"][rwg["tp"][m]]
        u = np.cross(t, nf)
        if (rwg["xyz"][rwg["pm"][m]] - a) @ u < 0:
            u = -u
        x[m] = J0 * u[0]
    perimeter = 2 * (size[1] + size[2])
    assert c @ x == pytest.approx(J0 * perimeter, rel=1e-12)
    assert np.sum(np.abs(c)) == pytest.approx(perimeter, rel=1e-12)


@pytest.mark.slow
def test_y_parameters_reciprocal():
    from synth import merge_meshes
    from oracle import operator as op
    from synth import box
    L, W, T = 60e-6, 10e-6, 5e-6
    bars = [box([0, 2 * W * i, 0], [L, 2 * W * i + W, T], [6, 2, 2]) for i in range(2)]
    xyz, tri, _ = merge_meshes(bars)
    prob = op.setup(xyz, tri, 2, (16, 8, 8), radius=3)
    ports = [([L / 2, 0, 0], [1, 0, 0], [-1, 2 * W * i - 1e-9, -1], [1, 2 * W * i + W + 1e-9, 1]) for i in range(2)]
    Ys = {}
    for f in (3e9, 3e10):
        Z = sibc.dense_efie_sibc(prob, f, 5.8e7, eps_bg=3.5)
        Y = sibc.y_parameters(Z, prob["rwg"], ports)
        # reciprocity, to the quadrature symmetry of the static near integrals
        assert np.abs(Y - Y.T).max() <= 1e-4 * np.abs(Y).max()
        Ys[f] = Y
    # electrically small gap dipoles: capacitive input admittance, Im Y proportional to f
    assert np.all(Ys[3e10].diagonal().imag > 0)
    ratio = Ys[3e10][0, 0].imag / Ys[3e9][0, 0].imag
    assert ratio == pytest.approx(10.0, rel=1e-2)
