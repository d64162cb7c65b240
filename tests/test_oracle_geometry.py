"""Pins for the oracle's RWG functions, quadrature, grid, anchors, weights and near list.

Each check compares against something other than the oracle code itself:
closed forms (triangle monomial integrals), RWG normalisation on the edge,
brute-force enumeration and independent polynomial integration.
"""

import math

import numpy as np
import pytest

from synth import icosphere, box
from oracle import rwg as rw, quadrature as qd, grid as gm


def test_icosphere_counts():
    for lev, nt in ((1, 80), (3, 1280)):
        xyz, tri = icosphere(lev)
        assert len(tri) == nt
        r = rw.build_rwg(xyz, tri)
        assert r["n"] == 3 * nt // 2            # closed surface: every edge interior
        assert len(xyz) - r["n"] + nt == 2      # Euler characteristic of a sphere


def test_rwg_edge_flux_and_divergence():
    """Normal component of f on its edge is +1 leaving T+ and entering T- (RWG normalisation)."""
    xyz, tri = icosphere(1)
    r = rw.build_rwg(xyz, tri)
    for n in range(r["n"]):
        a, b = xyz[r["ea"][n]], xyz[r["eb"][n]]
        mid = 0.5 * (a + b)
        for sgn, t, p in ((1, r["tp"][n], r["pp"][n]), (-1, r["tm"][n], r["pm"][n])):
            A = r["area"][t]
            c = r["length"][n] / (2 * A)
            f = sgn * c * (mid - xyz[p])
            # outward in-plane normal of the edge within triangle t
            nt_ = r["normal"][t]
            e = (b - a) / np.linalg.norm(b - a)
            m = np.cross(e, nt_)
            if np.dot(m, mid - xyz[p]) < 0:
                m = -m
            assert np.dot(f, m) == pytest.approx(sgn * 1.0, rel=1e-12)
        # total charge of one RWG is zero: (l/A+) A+ - (l/A-) A- = 0
        assert r["length"][n] - r["length"][n] == 0.0


def test_rwg_orientation_rule():
    """T+ traverses the edge from the smaller to the larger vertex id."""
    xyz, tri = icosphere(1)
    r = rw.build_rwg(xyz, tri)
    for n in range(r["n"]):
        a, b = r["ea"][n], r["eb"][n]
        assert a < b
        tv = list(tri[r["tp"][n]])
        i = tv.index(a)
        assert tv[(i + 1) % 3] == b


def test_mesh_errors():
    xyz, tri = icosphere(1)
    bad = np.concatenate([tri, tri[:1]])          # edge shared by three triangles
    with pytest.raises(rw.MeshError):
        rw.build_rwg(xyz, bad)
    flipped = tri.copy()
    flipped[0] = flipped[0][[0, 2, 1]]              # inconsistent orientation
    with pytest.raises(rw.MeshError):
        rw.build_rwg(xyz, flipped)
    degen = tri.copy()
    degen[0, 2] = degen[0, 1]
    with pytest.raises(rw.MeshError):
        rw.build_rwg(xyz, degen)


def test_triangle_rule_exact_monomials():
    """int_T l1^a l2^b l3^c dS = 2A a! b! c! / (a+b+c+2)!  for a+b+c <= 2q-2."""
    for q in (3, 5):
        bary, w = qd.triangle_rule(q)
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        for a in range(2 * q - 1):
            for b in range(2 * q - 1 - a):
                for c in range(2 * q - 1 - a - b):
                    num = np.sum(w * bary[:, 0] ** a * bary[:, 1] ** b * bary[:, 2] ** c)
                    exact = 2.0 * math.factorial(a) * math.factorial(b) * math.factorial(c) \
                        / math.factorial(a + b + c + 2)
                    assert num == pytest.approx(exact, rel=1e-12, abs=1e-16)


def test_anchor_is_nearest_node(small_sphere):
    """For order 2 the middle stencil node is the grid node nearest to the basis centre."""
    g = small_sphere["grid"]
    c = small_sphere["rwg"]["center"]
    anc = small_sphere["anc"]
    for a in range(3):
        nodes = g["origin"][a] + g["h"][a] * np.arange(g["n"][a])
        nearest = np.argmin(np.abs(c[:, a, None] - nodes[None, :]), axis=1)
        assert np.array_equal(anc[:, a] + 1, nearest)


def test_anchor_out_of_grid_raises():
    xyz, tri = icosphere(1)
    r = rw.build_rwg(xyz, tri)
    g = gm.make_grid(xyz, 2, [8, 8, 8])
    g2 = dict(g, origin=g["origin"] + 3 * g["h"])
    with pytest.raises(gm.GridError):
        gm.anchors(g2, r["center"])


def test_near_pairs_brute_force(small_sphere):
    anc = small_sphere["anc"]
    rp, cols = small_sphere["row_ptr"], small_sphere["cols"]
    N = len(anc)
    for m in range(N):
        brute = [n for n in range(N) if np.max(np.abs(anc[m] - anc[n])) <= 3]
        assert list(cols[rp[m]:rp[m + 1]]) == brute


def _exact_poly_moment(v0, v1, v2, A, field, alpha, r0, p_free, sgn, c, div):
    """int_T f_field(r) (r - r0)^alpha dS computed by expanding in barycentric monomials."""
    # (r - r0) = l1 (v0 - r0) + l2 (v1 - r0) + l3 (v2 - r0): expand product of linear forms
    P = np.stack([v0 - r0, v1 - r0, v2 - r0])       # [3 bary, 3 xyz]
    # polynomial in barycentrics as dict {(a,b,c): coef}
    poly = {(0, 0, 0): 1.0}

    def mul_linear(poly, coeffs):
        out = {}
        for (a, b, cc), v in poly.items():
            for i, k in enumerate(coeffs):
                key = (a + (i == 0), b + (i == 1), cc + (i == 2))
                out[key] = out.get(key, 0.0) + v * k
        return out

    for axis in range(3):
        for _ in range(alpha[axis]):
            poly = mul_linear(poly, P[:, axis])
    if field == 3:
        factor = {(0, 0, 0): div}
    else:
        q = np.stack([v0 - p_free, v1 - p_free, v2 - p_free])[:, field] * sgn * c
        factor = {(1, 0, 0): q[0], (0, 1, 0): q[1], (0, 0, 1): q[2]}
    tot = 0.0
    for (a, b, cc), v in poly.items():
        for (a2, b2, c2), w in factor.items():
            e = (a + a2, b + b2, cc + c2)
            tot += v * w * 2.0 * A * math.factorial(e[0]) * math.factorial(e[1]) \
                * math.factorial(e[2]) / math.factorial(sum(e) + 2)
    return tot


def test_projection_moment_matching(small_sphere):
    """sum_u Lambda_f[u,n] (r_u - r0)^alpha = int f (r - r0)^alpha dS for alpha_a <= n (moment matching: Sec. I and the opening of Sec. IV)."""
    r = small_sphere["rwg"]
    g = small_sphere["grid"]
    lam = small_sphere["lam"]
    anc = small_sphere["anc"]
    off = gm.stencil_offsets(2)
    xyz, tri = r["xyz"], r["tri"]
    for n in (0, 7, 31, 77):
        r0 = r["center"][n]
        nodes = g["origin"] + g["h"] * (anc[n] + off)          # [27,3]
        for alpha in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (2, 2, 2), (1, 1, 0), (0, 0, 2)]:
            lhs = np.einsum("uf,u->f", lam[n], np.prod((nodes - r0) ** np.array(alpha), axis=1))
            rhs = np.zeros(4)
            for sgn, t, p in ((1, r["tp"][n], r["pp"][n]), (-1, r["tm"][n], r["pm"][n])):
                A = r["area"][t]
                c = r["length"][n] / (2 * A)
                v = [xyz[tri[t, i]] for i in range(3)]
                for f in range(4):
                    rhs[f] += _exact_poly_moment(v[0], v[1], v[2], A, f, alpha, r0, xyz[p], sgn, c,
                                                 sgn * 2 * c)
            scale = np.abs(lam[n]).max() * np.max(np.abs(nodes - r0)) ** sum(alpha)
            assert np.allclose(lhs, rhs, rtol=0, atol=1e-12 * scale)


def test_charge_neutrality(small_sphere):
    lam = small_sphere["lam"]
    assert np.abs(lam[:, :, 3].sum(axis=1)).max() < 1e-12 * np.abs(lam[:, :, 3]).max()


def test_box_mesh_closed():
    xyz, tri = box([0, 0, 0], [3, 2, 1], [3, 2, 1])
    r = rw.build_rwg(xyz, tri)
    assert r["n"] == 3 * len(tri) // 2
    assert len(xyz) - r["n"] + len(tri) == 2


def test_flat_axis_takes_largest_spacing():
    """A planar mesh gets a usable spacing along its flat axis (the largest of the others)."""
    import numpy as np
    from oracle import grid as gridmod
    xyz = np.array([[0, 0, 0], [0.3, 0, 0], [0, 0.2, 0], [0.3, 0.2, 0.0]])
    g = gridmod.make_grid(xyz, 2, np.array([8, 8, 8]))
    assert g["h"][2] == max(g["h"][0], g["h"][1]) > 0
    assert g["origin"][2] == -g["margin"] * g["h"][2]
